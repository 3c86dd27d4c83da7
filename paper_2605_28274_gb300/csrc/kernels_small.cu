// Small-matrix side of the factorized methods, all in float64 on the device:
// the factored Sylvester operator (eq. 3.7), the inner products that give
// alpha, beta, omega, rho (eq. 3.6), the padded updates of X^, R^, P^ (and S^,
// T^), and the convergence test ||R^_{k+1}|| <= tol ||R^_0|| (Algorithms 4.1, 4.2).
//
// Small matrices are column-major with one fixed leading dimension and are
// zero outside their current extent, so each padding [M O; O O] of the
// algorithms is free: a kernel only ever writes inside the new extent.
// Reductions are deterministic: every CTA writes its partial sum, the last CTA
// to finish adds them in index order and updates the scalars in DevState.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace sylv {

namespace {

// ---------------------------------------------------------------- init
__global__ void init_small_kernel(DevState* st, double* hist, int s, int64_t lds, double* Rh, double* Ph,
                                  double* Rt, double* Uh, const double* __restrict__ RL,
                                  const double* __restrict__ RR, double tol) {
  // one CTA, thread 0 (s <= 8)
  if (threadIdx.x != 0) return;
  hist[0] = 1.0;
  if (st->status != ST_RUNNING) return;  // the QR of C1 or C2 already failed
  double nrm2 = 0.0;
  for (int t = 0; t < s; ++t)
    for (int u = 0; u < s; ++u) {
      double acc = 0.0;  // (R_L R_R^T)[u][t] = sum_c R_L[u][c] R_R[t][c]
      for (int c = 0; c < s; ++c) acc += RL[u + c * s] * RR[t + c * s];
      Rh[u + t * lds] = acc;
      Ph[u + t * lds] = acc;
      Rt[u + t * s] = acc;
      if (Uh) Uh[u + t * lds] = acc;  // CGS: U^_0 = R^_0
      nrm2 += acc * acc;
    }
  st->r0 = sqrt(nrm2);
  st->rnorm = st->r0;
  st->rho = nrm2;  // <R^_0, R^_0> (CG) = <R~_0, R^_0> (BiCGSTAB, R~_0 = R^_0)
  st->alpha = st->beta = st->omega = 0.0;
  st->tol = tol;
  st->iters = 0;
  st->exhausted[0] = st->exhausted[1] = 0;
  if (!isfinite(nrm2)) st->status = ST_NONFINITE;
  else if (nrm2 == 0.0) st->status = ST_CONVERGED;  // C1 C2^T = 0: X = 0
  else st->status = ST_RUNNING;
}

// ---------------------------------------------------------------- CG: Q^ for block tridiagonal H, G
// mode 0: Q^ = [H P^, 0] + [P^ G^T; 0]   (Sylvester)
// mode 1: M  = [H P^, 0]                 (Lyapunov, first half)
// mode 2: Q^ = M + M^T                   (Lyapunov, second half; Out is Q^, In is M)
// Modes 0 and 2 also reduce <P^, Q^(1:r,1:r)> and set alpha = rho / that (last CTA).
// cr = 0 (CG): the reduction <P^, Q^> sets alpha = rho / <P^, Q^>.  cr = 1 (CR: P is R^, Out
// is L(R)^): the reduction is rho_new = <R^, L(R)^>; with first it sets rho, otherwise
// beta = rho_new / rho and rho = rho_new.
__global__ void __launch_bounds__(NT) cg_q_kernel(DevState* st, int mode, int r, int s, const double* __restrict__ H,
                                                  const double* __restrict__ G, int64_t ldh,
                                                  const double* __restrict__ P, const double* __restrict__ In,
                                                  double* __restrict__ Out, int64_t lds, double* partials, int cr,
                                                  int first) {
  if (stopped(st)) return;
  __shared__ double sh[32];
  __shared__ int last_sh;
  const int rp = r + s;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  double pq = 0.0;
  if (a < rp) {
    double q = 0.0;
    if (mode == 2) {
      q = In[a + (int64_t)b * lds] + In[b + (int64_t)a * lds];
    } else {
      const int ba = a / s;
      if (b < r) {  // [H P^, 0]: H_{ba, c} nonzero for blocks ba-1..ba+1
        const int c0 = max(0, (ba - 1) * s), c1 = min(r, (ba + 2) * s);
        for (int c = c0; c < c1; ++c) q += H[a + (int64_t)c * ldh] * P[c + (int64_t)b * lds];
      }
      if (mode == 0 && a < r) {  // [P^ G^T; 0]
        const int bb = b / s;
        const int c0 = max(0, (bb - 1) * s), c1 = min(r, (bb + 2) * s);
        double q2 = 0.0;
        for (int c = c0; c < c1; ++c) q2 += P[a + (int64_t)c * lds] * G[b + (int64_t)c * ldh];
        q += q2;
      }
    }
    Out[a + (int64_t)b * lds] = q;
    if (a < r && b < r) pq = P[a + (int64_t)b * lds] * q;
  }
  if (mode == 1) return;
  pq = block_sum(pq, sh);
  const int bid = blockIdx.x + blockIdx.y * gridDim.x;
  if (threadIdx.x == 0) partials[bid] = pq;
  if (last_cta(&st->tickets[TK_CG_Q], &last_sh)) {
    const int nb = gridDim.x * gridDim.y;
    const double tot = cta_sum(partials, nb, 1, 0, sh);
    if (threadIdx.x == 0) {
      if (!isfinite(tot)) {
        st->status = ST_NONFINITE;
        st->breakdown_where = 1;
      } else if (cr) {
        if (tot == 0.0) {  // <R, L(R)> = 0: the CR recurrence breaks down
          st->status = ST_BREAKDOWN;
          st->breakdown_where = 20;
        } else {
          if (!first) st->beta = tot / st->rho;
          st->rho = tot;
        }
      } else if (!(tot > 0.0)) {  // <P, Q> <= 0: F not positive definite on this direction
        st->status = ST_BREAKDOWN;
        st->breakdown_where = 2;
      } else {
        st->alpha = st->rho / tot;
      }
    }
  }
}

// X^ <- pad(X^) + alpha P^ (extent r), R^ <- pad(R^) - alpha Q^ (extent r+s); then the
// test, rho_{k+1} = <R^,R^>, beta = rho_{k+1}/rho_k (last CTA).
// cr = 1: Q is L(P)^ and beta, rho come from the next operator application (cg_q_kernel, cr).
__global__ void __launch_bounds__(NT) cg_update_kernel(DevState* st, double* hist, int k, int r, int s,
                                                       double* __restrict__ X, double* __restrict__ R,
                                                       const double* __restrict__ P, const double* __restrict__ Q,
                                                       int64_t lds, double* partials, int cr) {
  if (stopped(st)) return;
  __shared__ double sh[32];
  __shared__ int last_sh;
  const int rp = r + s;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  const double alpha = st->alpha;
  double rr = 0.0;
  if (a < rp) {
    const int64_t i = a + (int64_t)b * lds;
    if (a < r && b < r) X[i] = X[i] + alpha * P[i];
    const double v = R[i] - alpha * Q[i];
    R[i] = v;
    rr = v * v;
  }
  rr = block_sum(rr, sh);
  const int bid = blockIdx.x + blockIdx.y * gridDim.x;
  if (threadIdx.x == 0) partials[bid] = rr;
  if (last_cta(&st->tickets[TK_CG_UPD], &last_sh)) {
    const int nb = gridDim.x * gridDim.y;
    const double tot = cta_sum(partials, nb, 1, 0, sh);
    if (threadIdx.x == 0) {
      const double rn = sqrt(tot);
      hist[k + 1] = rn / st->r0;
      st->rnorm = rn;
      st->iters = k + 1;
      if (!isfinite(rn)) {
        st->status = ST_NONFINITE;
        st->breakdown_where = 3;
      } else if (rn <= st->r0 * st->tol) {
        st->status = ST_CONVERGED;
      } else if (!cr) {
        st->beta = tot / st->rho;
        st->rho = tot;
      }
    }
  }
}

// CR: P^ <- R^ + beta pad(P^), L(P)^ <- L(R)^ + beta pad(L(P)^) over extent rpp, then
// alpha = rho / <L(P)^, L(P)^> (last CTA).
__global__ void __launch_bounds__(NT) cr_p_kernel(DevState* st, int rpp, double* __restrict__ P,
                                                  double* __restrict__ LP, const double* __restrict__ R,
                                                  const double* __restrict__ LR, int64_t lds, double* partials) {
  if (stopped(st)) return;
  __shared__ double sh[32];
  __shared__ int last_sh;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  const double beta = st->beta;
  double qq = 0.0;
  if (a < rpp) {
    const int64_t i = a + (int64_t)b * lds;
    P[i] = R[i] + beta * P[i];
    const double v = LR[i] + beta * LP[i];
    LP[i] = v;
    qq = v * v;
  }
  qq = block_sum(qq, sh);
  const int bid = blockIdx.x + blockIdx.y * gridDim.x;
  if (threadIdx.x == 0) partials[bid] = qq;
  if (last_cta(&st->tickets[TK_CG_Q], &last_sh)) {
    const int nb = gridDim.x * gridDim.y;
    const double tot = cta_sum(partials, nb, 1, 0, sh);
    if (threadIdx.x == 0) {
      if (!isfinite(tot)) {
        st->status = ST_NONFINITE;
        st->breakdown_where = 21;
      } else if (tot == 0.0) {
        st->status = ST_BREAKDOWN;
        st->breakdown_where = 22;
      } else {
        st->alpha = st->rho / tot;
      }
    }
  }
}

// P^ <- R^ + beta pad(P^) over extent rp.
__global__ void __launch_bounds__(NT) cg_p_kernel(const DevState* st, int rp, double* __restrict__ P,
                                                  const double* __restrict__ R, int64_t lds) {
  if (stopped(st)) return;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  if (a >= rp) return;
  const int64_t i = a + (int64_t)b * lds;
  P[i] = R[i] + st->beta * P[i];
}

// ---------------------------------------------------------------- BiCGSTAB: dense factored operator
// Out = [H Z, 0] + [Z G^T; 0] for Z with extent r (H, G block upper Hessenberg,
// (r+s) x r).  32 x 32 output tiles, 32-deep k-slices in shared memory, 2 x 2
// outputs per thread; k-slices left of the Hessenberg band of a tile are skipped.
// The skipping makes tiles unequal (the top-left tile does the most work), so the
// tiles are small enough that the block scheduler keeps every SM busy.
// With OMEGA, the tile also reduces <Out(1:r,1:r), Z> and <Out, Out> and the last
// CTA sets omega (Algorithm 4.2).
constexpr int GBM = 32, GBK = 32;

template <bool OMEGA>
__global__ void __launch_bounds__(NT) sylv_gemm_kernel(DevState* st, int r, int s, const double* __restrict__ H,
                                                       const double* __restrict__ G, int64_t ldh,
                                                       const double* __restrict__ Z, double* __restrict__ Out,
                                                       int64_t lds, double* partials) {
  if (stopped(st)) return;
  __shared__ double As[GBK][GBM + 1];
  __shared__ double Bs[GBK][GBM + 1];
  __shared__ double sh[32];
  __shared__ int last_sh;
  const int rp = r + s;
  const int a0 = blockIdx.x * GBM, b0 = blockIdx.y * GBM;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};

  // term 1: (H Z)[a][b] for b < r
  if (b0 < r) {
    const int clo = max(0, (a0 / s - 1) * s);
    for (int c0 = clo; c0 < r; c0 += GBK) {
      for (int e = threadIdx.x; e < GBK * GBM; e += NT) {
        const int aa = e % GBM, kk = e / GBM;  // H column-major: contiguous in a
        const int a = a0 + aa, c = c0 + kk;
        As[kk][aa] = (a < rp && c < r) ? H[a + (int64_t)c * ldh] : 0.0;
        const int kk2 = e % GBK, bb = e / GBK;  // Z column-major: contiguous in c
        const int c2 = c0 + kk2, b = b0 + bb;
        Bs[kk2][bb] = (c2 < r && b < r) ? Z[c2 + (int64_t)b * lds] : 0.0;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < GBK; ++kk) {
        const double a_0 = As[kk][tx], a_1 = As[kk][tx + 16];
        const double b_0 = Bs[kk][ty], b_1 = Bs[kk][ty + 16];
        acc[0][0] += a_0 * b_0;
        acc[0][1] += a_0 * b_1;
        acc[1][0] += a_1 * b_0;
        acc[1][1] += a_1 * b_1;
      }
      __syncthreads();
    }
  }
  // term 2: (Z G^T)[a][b] for a < r
  if (a0 < r) {
    const int clo = max(0, (b0 / s - 1) * s);
    for (int c0 = clo; c0 < r; c0 += GBK) {
      for (int e = threadIdx.x; e < GBK * GBM; e += NT) {
        const int aa = e % GBM, kk = e / GBM;
        const int a = a0 + aa, c = c0 + kk;
        As[kk][aa] = (a < r && c < r) ? Z[a + (int64_t)c * lds] : 0.0;
        const int b = b0 + aa;  // G^T[c][b] = G[b][c]: contiguous in b
        Bs[kk][aa] = (b < rp && c < r) ? G[b + (int64_t)c * ldh] : 0.0;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < GBK; ++kk) {
        const double a_0 = As[kk][tx], a_1 = As[kk][tx + 16];
        const double b_0 = Bs[kk][ty], b_1 = Bs[kk][ty + 16];
        acc[0][0] += a_0 * b_0;
        acc[0][1] += a_0 * b_1;
        acc[1][0] += a_1 * b_0;
        acc[1][1] += a_1 * b_1;
      }
      __syncthreads();
    }
  }
  double ts = 0.0, tt = 0.0;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int a = a0 + tx + 16 * i, b = b0 + ty + 16 * j;
      if (a < rp && b < rp) {
        Out[a + (int64_t)b * lds] = acc[i][j];
        if (OMEGA) {
          tt += acc[i][j] * acc[i][j];
          if (a < r && b < r) ts += acc[i][j] * Z[a + (int64_t)b * lds];
        }
      }
    }
  if (!OMEGA) return;
  ts = block_sum(ts, sh);
  tt = block_sum(tt, sh);
  const int bid = blockIdx.x + blockIdx.y * gridDim.x;
  if (threadIdx.x == 0) {
    partials[2 * bid] = ts;
    partials[2 * bid + 1] = tt;
  }
  if (last_cta(&st->tickets[TK_BI_T], &last_sh)) {
    const int nb = gridDim.x * gridDim.y;
    const double s1 = cta_sum(partials, nb, 2, 0, sh), s2 = cta_sum(partials, nb, 2, 1, sh);
    if (threadIdx.x == 0) {
      if (!isfinite(s1) || !isfinite(s2)) {
        st->status = ST_NONFINITE;
        st->breakdown_where = 4;
      } else if (s2 == 0.0 || s1 == 0.0) {  // T = 0 or omega = 0
        st->status = ST_BREAKDOWN;
        st->breakdown_where = 5;
      } else {
        st->omega = s1 / s2;
      }
    }
  }
}

// Double-float variant of sylv_gemm_kernel for the mixed-precision mode: operands are
// split into hi + lo floats as they are staged in shared memory, products use the
// error-free FMA product and sums the error-free two-sum (Dekker 1971), so the
// accumulation runs on the FP32 pipes with a unit roundoff of about 2^-48 (the
// mixed mode's factors are FP32, 2^-24).  Same tiling, Hessenberg skipping and
// omega reduction as the float64 kernel.
struct dfp {
  float hi, lo;
};

__device__ __forceinline__ dfp dsplit(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ void dfma2(dfp& acc, dfp u, dfp y) {
  const float ph = __fmul_rn(u.hi, y.hi);
  float pl = __fmaf_rn(u.hi, y.hi, -ph);
  pl = __fmaf_rn(u.hi, y.lo, pl);
  pl = __fmaf_rn(u.lo, y.hi, pl);
  const float s = __fadd_rn(acc.hi, ph);
  const float bb = __fsub_rn(s, acc.hi);
  const float e = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(ph, bb));
  const float t = __fadd_rn(__fadd_rn(e, acc.lo), pl);
  acc.hi = __fadd_rn(s, t);
  acc.lo = __fsub_rn(t, __fsub_rn(acc.hi, s));
}

// Hi/lo split of the columns [c0, c1) of a column-major matrix (rows 0..rows-1, ld ld).
__global__ void __launch_bounds__(NT) split_cols_kernel(const DevState* st, int rows, int c0, int c1,
                                                        const double* __restrict__ M, int64_t ld,
                                                        dfp* __restrict__ out) {
  if (stopped(st)) return;
  const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (e >= (int64_t)rows * (c1 - c0)) return;
  const int a = (int)(e % rows);
  const int64_t c = c0 + e / rows;
  out[a + c * ld] = dsplit(M[a + c * ld]);
}

// The operands arrive split (Hs, Gs, Zs: the hi/lo pairs of H, G, Z, same layouts), so
// the inner loop runs on the FP32 pipes only; Z itself is read for the omega sums.
template <bool OMEGA>
__global__ void __launch_bounds__(NT) sylv_gemm_df_kernel(DevState* st, int r, int s, const dfp* __restrict__ Hs,
                                                          const dfp* __restrict__ Gs, int64_t ldh,
                                                          const dfp* __restrict__ Zs, const double* __restrict__ Z,
                                                          double* __restrict__ Out, int64_t lds, double* partials) {
  if (stopped(st)) return;
  __shared__ dfp As[GBK][GBM + 1];
  __shared__ dfp Bs[GBK][GBM + 1];
  __shared__ double sh[32];
  __shared__ int last_sh;
  const int rp = r + s;
  const int a0 = blockIdx.x * GBM, b0 = blockIdx.y * GBM;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  dfp acc[2][2] = {{{0.f, 0.f}, {0.f, 0.f}}, {{0.f, 0.f}, {0.f, 0.f}}};
  if (b0 < r) {  // (H Z)[a][b], b < r
    const int clo = max(0, (a0 / s - 1) * s);
    for (int c0 = clo; c0 < r; c0 += GBK) {
      for (int e = threadIdx.x; e < GBK * GBM; e += NT) {
        const int aa = e % GBM, kk = e / GBM;
        const int a = a0 + aa, c = c0 + kk;
        As[kk][aa] = (a < rp && c < r) ? Hs[a + (int64_t)c * ldh] : dfp{0.0f, 0.0f};
        const int kk2 = e % GBK, bb = e / GBK;
        const int c2 = c0 + kk2, b = b0 + bb;
        Bs[kk2][bb] = (c2 < r && b < r) ? Zs[c2 + (int64_t)b * lds] : dfp{0.0f, 0.0f};
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < GBK; ++kk) {
        const dfp a_0 = As[kk][tx], a_1 = As[kk][tx + 16];
        const dfp b_0 = Bs[kk][ty], b_1 = Bs[kk][ty + 16];
        dfma2(acc[0][0], a_0, b_0);
        dfma2(acc[0][1], a_0, b_1);
        dfma2(acc[1][0], a_1, b_0);
        dfma2(acc[1][1], a_1, b_1);
      }
      __syncthreads();
    }
  }
  if (a0 < r) {  // (Z G^T)[a][b], a < r
    const int clo = max(0, (b0 / s - 1) * s);
    for (int c0 = clo; c0 < r; c0 += GBK) {
      for (int e = threadIdx.x; e < GBK * GBM; e += NT) {
        const int aa = e % GBM, kk = e / GBM;
        const int a = a0 + aa, c = c0 + kk;
        As[kk][aa] = (a < r && c < r) ? Zs[a + (int64_t)c * lds] : dfp{0.0f, 0.0f};
        const int b = b0 + aa;
        Bs[kk][aa] = (b < rp && c < r) ? Gs[b + (int64_t)c * ldh] : dfp{0.0f, 0.0f};
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < GBK; ++kk) {
        const dfp a_0 = As[kk][tx], a_1 = As[kk][tx + 16];
        const dfp b_0 = Bs[kk][ty], b_1 = Bs[kk][ty + 16];
        dfma2(acc[0][0], a_0, b_0);
        dfma2(acc[0][1], a_0, b_1);
        dfma2(acc[1][0], a_1, b_0);
        dfma2(acc[1][1], a_1, b_1);
      }
      __syncthreads();
    }
  }
  double ts = 0.0, tt = 0.0;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int a = a0 + tx + 16 * i, b = b0 + ty + 16 * j;
      if (a < rp && b < rp) {
        const double v = (double)acc[i][j].hi + (double)acc[i][j].lo;
        Out[a + (int64_t)b * lds] = v;
        if (OMEGA) {
          tt += v * v;
          if (a < r && b < r) ts += v * Z[a + (int64_t)b * lds];
        }
      }
    }
  if (!OMEGA) return;
  ts = block_sum(ts, sh);
  tt = block_sum(tt, sh);
  const int bid = blockIdx.x + blockIdx.y * gridDim.x;
  if (threadIdx.x == 0) {
    partials[2 * bid] = ts;
    partials[2 * bid + 1] = tt;
  }
  if (last_cta(&st->tickets[TK_BI_T], &last_sh)) {
    const int nb = gridDim.x * gridDim.y;
    const double s1 = cta_sum(partials, nb, 2, 0, sh), s2 = cta_sum(partials, nb, 2, 1, sh);
    if (threadIdx.x == 0) {
      if (!isfinite(s1) || !isfinite(s2)) {
        st->status = ST_NONFINITE;
        st->breakdown_where = 4;
      } else if (s2 == 0.0 || s1 == 0.0) {
        st->status = ST_BREAKDOWN;
        st->breakdown_where = 5;
      } else {
        st->omega = s1 / s2;
      }
    }
  }
}

// alpha_k = rho_k / <R~_0, Q^(1:s,1:s)>  (one CTA)
__global__ void bicg_alpha_kernel(DevState* st, int s, const double* __restrict__ Rt, const double* __restrict__ Q,
                                  int64_t lds) {
  if (stopped(st)) return;
  if (threadIdx.x != 0) return;
  double d = 0.0;
  for (int t = 0; t < s; ++t)
    for (int u = 0; u < s; ++u) d += Rt[u + t * s] * Q[u + (int64_t)t * lds];
  if (!isfinite(d)) {
    st->status = ST_NONFINITE;
    st->breakdown_where = 6;
  } else if (d == 0.0) {
    st->status = ST_BREAKDOWN;
    st->breakdown_where = 7;
  } else {
    st->alpha = st->rho / d;
  }
}

// S^ = pad(R^) - alpha Q^ over extent rp
__global__ void __launch_bounds__(NT) bicg_s_kernel(const DevState* st, int rp, double* __restrict__ S,
                                                    const double* __restrict__ R, const double* __restrict__ Q,
                                                    int64_t lds) {
  if (stopped(st)) return;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  if (a >= rp) return;
  const int64_t i = a + (int64_t)b * lds;
  S[i] = R[i] - st->alpha * Q[i];
}

// X^ <- pad(X^) + pad(alpha P^) + omega S^ (extent rp); R^ <- pad(S^) - omega T^ (extent rpp);
// then the test, rho_{k+1} = <R~_0, R^(1:s,1:s)>, beta = (alpha/omega)(rho_{k+1}/rho_k).
__global__ void __launch_bounds__(NT) bicg_update_kernel(DevState* st, double* hist, int k, int rp, int rpp, int s,
                                                         double* __restrict__ X, double* __restrict__ R,
                                                         const double* __restrict__ P,
                                                         const double* __restrict__ S,
                                                         const double* __restrict__ T, const double* __restrict__ Rt,
                                                         int64_t lds, double* partials) {
  if (stopped(st)) return;
  __shared__ double sh[32];
  __shared__ int last_sh;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  const double alpha = st->alpha, omega = st->omega;
  double rr = 0.0;
  if (a < rpp) {
    const int64_t i = a + (int64_t)b * lds;
    if (a < rp && b < rp) X[i] = X[i] + alpha * P[i] + omega * S[i];
    const double v = S[i] - omega * T[i];
    R[i] = v;
    rr = v * v;
  }
  rr = block_sum(rr, sh);
  const int bid = blockIdx.x + blockIdx.y * gridDim.x;
  if (threadIdx.x == 0) partials[bid] = rr;
  if (last_cta(&st->tickets[TK_BI_UPD], &last_sh)) {
    const int nb = gridDim.x * gridDim.y;
    const double tot = cta_sum(partials, nb, 1, 0, sh);
    if (threadIdx.x == 0) {
      const double rn = sqrt(tot);
      hist[k + 1] = rn / st->r0;
      st->rnorm = rn;
      st->iters = k + 1;
      if (!isfinite(rn)) {
        st->status = ST_NONFINITE;
        st->breakdown_where = 8;
      } else if (rn <= st->r0 * st->tol) {
        st->status = ST_CONVERGED;
      } else {
        double rho_new = 0.0;
        for (int t = 0; t < s; ++t)
          for (int u = 0; u < s; ++u) rho_new += Rt[u + t * s] * __ldcg(R + u + (int64_t)t * lds);
        if (rho_new == 0.0) {
          st->status = ST_BREAKDOWN;
          st->breakdown_where = 9;
        } else {
          st->beta = (alpha / omega) * (rho_new / st->rho);
          st->rho = rho_new;
        }
      }
    }
  }
}

// P^ <- R^ + beta (pad(P^) - omega pad(Q^)) over extent rpp
__global__ void __launch_bounds__(NT) bicg_p_kernel(const DevState* st, int rpp, double* __restrict__ P,
                                                    const double* __restrict__ R, const double* __restrict__ Q,
                                                    int64_t lds) {
  if (stopped(st)) return;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  if (a >= rpp) return;
  const int64_t i = a + (int64_t)b * lds;
  P[i] = R[i] + st->beta * (P[i] - st->omega * Q[i]);
}

// ---------------------------------------------------------------- factorized CGS
// The CGS recurrence on padded small matrices (eq. 3.5), inner products with R~_0 on the
// leading s x s block (eq. 3.6); alpha = rho / <R~_0, V^(1:s,1:s)> comes from
// bicg_alpha_kernel with V^ = L(P^) in the Q^ buffer.
//
// Q^ = pad(U^) - alpha V^ (in place, V -> Q), W^ = pad(U^) + Q^, X^ <- pad(X^) + alpha W^,
// over extent rp = (2k+2)s.
__global__ void __launch_bounds__(NT) cgs_q_kernel(const DevState* st, int rp, double* __restrict__ X,
                                                   const double* __restrict__ U, double* __restrict__ VQ,
                                                   double* __restrict__ W, int64_t lds) {
  if (stopped(st)) return;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  if (a >= rp) return;
  const int64_t i = a + (int64_t)b * lds;
  const double alpha = st->alpha;
  const double u = U[i];
  const double q = u - alpha * VQ[i];
  const double w = u + q;
  VQ[i] = q;
  W[i] = w;
  X[i] = X[i] + alpha * w;
}

// R^ <- pad(R^) - alpha T^ over extent rpp = (2k+3)s (T^ = L(W^)); then the test,
// rho_{k+1} = <R~_0, R^(1:s,1:s)> and beta = rho_{k+1} / rho_k (last CTA).
__global__ void __launch_bounds__(NT) cgs_update_kernel(DevState* st, double* hist, int k, int rpp, int s,
                                                        double* __restrict__ R, const double* __restrict__ T,
                                                        const double* __restrict__ Rt, int64_t lds,
                                                        double* partials) {
  if (stopped(st)) return;
  __shared__ double sh[32];
  __shared__ int last_sh;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  const double alpha = st->alpha;
  double rr = 0.0;
  if (a < rpp) {
    const int64_t i = a + (int64_t)b * lds;
    const double v = R[i] - alpha * T[i];
    R[i] = v;
    rr = v * v;
  }
  rr = block_sum(rr, sh);
  const int bid = blockIdx.x + blockIdx.y * gridDim.x;
  if (threadIdx.x == 0) partials[bid] = rr;
  if (last_cta(&st->tickets[TK_BI_UPD], &last_sh)) {
    const int nb = gridDim.x * gridDim.y;
    const double tot = cta_sum(partials, nb, 1, 0, sh);
    if (threadIdx.x == 0) {
      const double rn = sqrt(tot);
      hist[k + 1] = rn / st->r0;
      st->rnorm = rn;
      st->iters = k + 1;
      if (!isfinite(rn)) {
        st->status = ST_NONFINITE;
        st->breakdown_where = 8;
      } else if (rn <= st->r0 * st->tol) {
        st->status = ST_CONVERGED;
      } else {
        double rho_new = 0.0;
        for (int t = 0; t < s; ++t)
          for (int u = 0; u < s; ++u) rho_new += Rt[u + t * s] * __ldcg(R + u + (int64_t)t * lds);
        if (rho_new == 0.0) {
          st->status = ST_BREAKDOWN;
          st->breakdown_where = 9;
        } else {
          st->beta = rho_new / st->rho;
          st->rho = rho_new;
        }
      }
    }
  }
}

// U^ <- R^ + beta pad(Q^);  P^ <- U^ + beta (pad(Q^) + beta pad(P^))  over extent rpp.
__global__ void __launch_bounds__(NT) cgs_p_kernel(const DevState* st, int rpp, double* __restrict__ U,
                                                   double* __restrict__ P, const double* __restrict__ R,
                                                   const double* __restrict__ Q, int64_t lds) {
  if (stopped(st)) return;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  if (a >= rpp) return;
  const int64_t i = a + (int64_t)b * lds;
  const double beta = st->beta;
  const double q = Q[i];
  const double u = R[i] + beta * q;
  U[i] = u;
  P[i] = u + beta * (q + beta * P[i]);
}

// ---------------------------------------------------------------- factorized GPBiCG
// The GPBiCG recurrence on padded small matrices (eq. 3.5; <R~_0, .> on the leading s x s
// block, eq. 3.6), with extents e1 = (2k+1)s (P^, R^), e2 = e1 + s (L(P)^, T^, Y^, U^, Z^, X^)
// and e3 = e2 + s (L(T)^, W^, new R^).  zeta lives in DevState::omega, eta in DevState::eta.

// P^ <- R^ + beta (P^ - U^) over extent e1.
__global__ void __launch_bounds__(NT) gp_p_kernel(const DevState* st, int e1, double* __restrict__ P,
                                                  const double* __restrict__ R, const double* __restrict__ U,
                                                  int64_t lds) {
  if (stopped(st)) return;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  if (a >= e1) return;
  const int64_t i = a + (int64_t)b * lds;
  P[i] = R[i] + st->beta * (P[i] - U[i]);
}

// Y^ <- T_prev^ - R^ - alpha W^ + alpha L(P)^,  T^ <- R^ - alpha L(P)^  over extent e2.
__global__ void __launch_bounds__(NT) gp_ty_kernel(const DevState* st, int e2, double* __restrict__ Y,
                                                   double* __restrict__ T, const double* __restrict__ Tp,
                                                   const double* __restrict__ R, const double* __restrict__ W,
                                                   const double* __restrict__ LP, int64_t lds) {
  if (stopped(st)) return;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  if (a >= e2) return;
  const int64_t i = a + (int64_t)b * lds;
  const double alpha = st->alpha, lp = LP[i], r = R[i];
  Y[i] = Tp[i] - r - alpha * W[i] + alpha * lp;
  T[i] = r - alpha * lp;
}

// zeta, eta minimise ||T - zeta L(T) - eta Y||: the five inner products <Y,Y>, <L(T),T>,
// <Y,T>, <L(T),Y> (extent e2) and <L(T),L(T)> (extent e3), per-CTA partials summed in CTA
// order by the last CTA.  The first iteration has eta = 0 (zeta = <L(T),T> / <L(T),L(T)>).
__global__ void __launch_bounds__(NT) gp_zeta_kernel(DevState* st, int k, int e2, int e3,
                                                     const double* __restrict__ Y, const double* __restrict__ T,
                                                     const double* __restrict__ LT, int64_t lds,
                                                     double* __restrict__ part) {
  if (stopped(st)) return;
  __shared__ double sh[32];
  __shared__ int last_sh;
  double yy = 0.0, tt = 0.0, yt = 0.0, ty = 0.0, aa = 0.0;
  const int64_t E = (int64_t)e3 * e3;
  for (int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x; q < E; q += (int64_t)gridDim.x * NT) {
    const int a = (int)(q % e3), b = (int)(q / e3);
    const int64_t i = a + (int64_t)b * lds;
    const double lt = LT[i];
    aa += lt * lt;
    if (a < e2 && b < e2) {
      const double y = Y[i], t = T[i];
      yy += y * y;
      tt += lt * t;
      yt += y * t;
      ty += lt * y;
    }
  }
  yy = block_sum(yy, sh);
  tt = block_sum(tt, sh);
  yt = block_sum(yt, sh);
  ty = block_sum(ty, sh);
  aa = block_sum(aa, sh);
  if (threadIdx.x == 0) {
    double* o = part + 5 * (int64_t)blockIdx.x;
    o[0] = yy;
    o[1] = tt;
    o[2] = yt;
    o[3] = ty;
    o[4] = aa;
  }
  if (last_cta(&st->tickets[TK_GP_ZETA], &last_sh)) {
    double v[5];
    for (int j = 0; j < 5; ++j) v[j] = cta_sum(part, (int)gridDim.x, 5, j, sh);
    if (threadIdx.x == 0) {
      double zeta, eta;
      if (k == 0) {
        zeta = v[1] / v[4];
        eta = 0.0;
      } else {
        const double den = v[4] * v[0] - v[3] * v[3];
        zeta = (v[0] * v[1] - v[2] * v[3]) / den;
        eta = (v[4] * v[2] - v[3] * v[1]) / den;
      }
      if (!isfinite(zeta) || !isfinite(eta)) {
        st->status = ST_NONFINITE;
        st->breakdown_where = 30;
      } else if (zeta == 0.0) {
        st->status = ST_BREAKDOWN;
        st->breakdown_where = 31;
      } else {
        st->omega = zeta;
        st->eta = eta;
      }
    }
  }
}

// With the old beta, U^, Z^, R^: U^ <- zeta L(P)^ + eta (T_prev^ - R^ + beta U^), Z^ <- zeta R^ +
// eta Z^ - alpha U^, X^ <- X^ + alpha P^ + Z^ (extent e2); R^ <- T^ - eta Y^ - zeta L(T)^ (e3);
// then the test, rho_{k+1} = <R~_0, R^(1:s,1:s)> and beta = (alpha / zeta) rho_{k+1} / rho_k.
__global__ void __launch_bounds__(NT) gp_update_kernel(DevState* st, double* hist, int k, int e2, int e3, int s,
                                                       double* __restrict__ X, double* __restrict__ R,
                                                       double* __restrict__ U, double* __restrict__ Z,
                                                       const double* __restrict__ P, const double* __restrict__ LP,
                                                       const double* __restrict__ Tp, const double* __restrict__ T,
                                                       const double* __restrict__ Y, const double* __restrict__ LT,
                                                       const double* __restrict__ Rt, int64_t lds,
                                                       double* partials) {
  if (stopped(st)) return;
  __shared__ double sh[32];
  __shared__ int last_sh;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  const double alpha = st->alpha, beta = st->beta, zeta = st->omega, eta = st->eta;
  double rr = 0.0;
  if (a < e3) {
    const int64_t i = a + (int64_t)b * lds;
    const double r_old = R[i];
    if (a < e2 && b < e2) {
      const double u = zeta * LP[i] + eta * (Tp[i] - r_old + beta * U[i]);
      const double z = zeta * r_old + eta * Z[i] - alpha * u;
      U[i] = u;
      Z[i] = z;
      X[i] = X[i] + alpha * P[i] + z;
    }
    const double v = T[i] - eta * Y[i] - zeta * LT[i];
    R[i] = v;
    rr = v * v;
  }
  rr = block_sum(rr, sh);
  const int bid = blockIdx.x + blockIdx.y * gridDim.x;
  if (threadIdx.x == 0) partials[bid] = rr;
  if (last_cta(&st->tickets[TK_BI_UPD], &last_sh)) {
    const int nb = gridDim.x * gridDim.y;
    const double tot = cta_sum(partials, nb, 1, 0, sh);
    if (threadIdx.x == 0) {
      const double rn = sqrt(tot);
      hist[k + 1] = rn / st->r0;
      st->rnorm = rn;
      st->iters = k + 1;
      if (!isfinite(rn)) {
        st->status = ST_NONFINITE;
        st->breakdown_where = 32;
      } else if (rn <= st->r0 * st->tol) {
        st->status = ST_CONVERGED;
      } else {
        double rho_new = 0.0;
        for (int t = 0; t < s; ++t)
          for (int u = 0; u < s; ++u) rho_new += Rt[u + t * s] * __ldcg(R + u + (int64_t)t * lds);
        if (rho_new == 0.0) {
          st->status = ST_BREAKDOWN;
          st->breakdown_where = 33;
        } else {
          st->beta = (alpha / zeta) * (rho_new / st->rho);
          st->rho = rho_new;
        }
      }
    }
  }
}

// W^ <- L(T)^ + beta L(P)^, T_prev^ <- T^  over extent e3 (the new beta).
__global__ void __launch_bounds__(NT) gp_w_kernel(const DevState* st, int e3, double* __restrict__ W,
                                                  double* __restrict__ Tp, const double* __restrict__ LT,
                                                  const double* __restrict__ LP, const double* __restrict__ T,
                                                  int64_t lds) {
  if (stopped(st)) return;
  const int a = blockIdx.x * NT + threadIdx.x;
  const int b = blockIdx.y;
  if (a >= e3) return;
  const int64_t i = a + (int64_t)b * lds;
  W[i] = LT[i] + st->beta * LP[i];
  Tp[i] = T[i];
}

dim3 elem_grid(int rows, int cols) { return dim3((unsigned)((rows + NT - 1) / NT), (unsigned)cols); }

}  // namespace

void launch_init_small(cudaStream_t strm, const SmallCtx& c, const double* RL, const double* RR, double tol,
                       bool cgs) {
  init_small_kernel<<<counted(1), 32, 0, strm>>>(c.st, c.hist, c.s, c.lds, c.Rh, c.Ph, c.Rt, cgs ? c.Uh : nullptr,
                                                 RL, RR, tol);
}

void launch_cgs_q(cudaStream_t strm, const SmallCtx& c, int rp) {
  cgs_q_kernel<<<counted(elem_grid(rp, rp)), NT, 0, strm>>>(c.st, rp, c.Xh, c.Uh, c.Qh, c.Th, c.lds);
}

void launch_cgs_update(cudaStream_t strm, const SmallCtx& c, int k, int rpp) {
  cgs_update_kernel<<<counted(elem_grid(rpp, rpp)), NT, 0, strm>>>(c.st, c.hist, k, rpp, c.s, c.Rh, c.Sh, c.Rt,
                                                                   c.lds, c.partials);
}

void launch_gp_p(cudaStream_t strm, const SmallCtx& c, int e1) {
  gp_p_kernel<<<counted(elem_grid(e1, e1)), NT, 0, strm>>>(c.st, e1, c.Ph, c.Rh, c.Uh, c.lds);
}

void launch_gp_ty(cudaStream_t strm, const SmallCtx& c, int e2) {
  gp_ty_kernel<<<counted(elem_grid(e2, e2)), NT, 0, strm>>>(c.st, e2, c.gY, c.Th, c.gTp, c.Rh, c.gW, c.Qh, c.lds);
}

void launch_gp_zeta(cudaStream_t strm, const SmallCtx& c, int k, int e2) {
  const int e3 = e2 + c.s;
  const int64_t E = (int64_t)e3 * e3;
  const unsigned g = (unsigned)std::min<int64_t>((E + NT - 1) / NT, GP_ZETA_CTAS);
  gp_zeta_kernel<<<counted(g), NT, 0, strm>>>(c.st, k, e2, e3, c.gY, c.Th, c.Sh, c.lds, c.gPart);
}

void launch_gp_update(cudaStream_t strm, const SmallCtx& c, int k, int e2) {
  const int e3 = e2 + c.s;
  gp_update_kernel<<<counted(elem_grid(e3, e3)), NT, 0, strm>>>(c.st, c.hist, k, e2, e3, c.s, c.Xh, c.Rh, c.Uh,
                                                                c.gZ, c.Ph, c.Qh, c.gTp, c.Th, c.gY, c.Sh, c.Rt,
                                                                c.lds, c.partials);
}

void launch_gp_w(cudaStream_t strm, const SmallCtx& c, int e3) {
  gp_w_kernel<<<counted(elem_grid(e3, e3)), NT, 0, strm>>>(c.st, e3, c.gW, c.gTp, c.Sh, c.Qh, c.Th, c.lds);
}

void launch_cgs_p(cudaStream_t strm, const SmallCtx& c, int rpp) {
  cgs_p_kernel<<<counted(elem_grid(rpp, rpp)), NT, 0, strm>>>(c.st, rpp, c.Uh, c.Ph, c.Rh, c.Qh, c.lds);
}

void launch_cg_q(cudaStream_t strm, const SmallCtx& c, int mode, int r) {
  const int rp = r + c.s;
  double* out = mode == 1 ? c.Th : c.Qh;  // Lyapunov: the T^ buffer holds M = [H P^, 0]
  cg_q_kernel<<<counted(elem_grid(rp, rp)), NT, 0, strm>>>(c.st, mode, r, c.s, c.H, c.G, c.ldh, c.Ph, c.Th, out, c.lds,
                                                  c.partials, 0, 0);
}

void launch_cr_op(cudaStream_t strm, const SmallCtx& c, int mode, int r, bool first) {
  const int rp = r + c.s;
  double* out = mode == 1 ? c.Th : c.Sh;  // L(R)^ in the S^ buffer (Lyapunov: M in T^ first)
  cg_q_kernel<<<counted(elem_grid(rp, rp)), NT, 0, strm>>>(c.st, mode, r, c.s, c.H, c.G, c.ldh, c.Rh, c.Th, out, c.lds,
                                                  c.partials, 1, first ? 1 : 0);
}

void launch_cr_p(cudaStream_t strm, const SmallCtx& c, int rpp) {
  cr_p_kernel<<<counted(elem_grid(rpp, rpp)), NT, 0, strm>>>(c.st, rpp, c.Ph, c.Qh, c.Rh, c.Sh, c.lds, c.partials);
}

void launch_cg_update(cudaStream_t strm, const SmallCtx& c, int k, int r, bool cr) {
  const int rp = r + c.s;
  cg_update_kernel<<<counted(elem_grid(rp, rp)), NT, 0, strm>>>(c.st, c.hist, k, r, c.s, c.Xh, c.Rh, c.Ph, c.Qh, c.lds,
                                                       c.partials, cr ? 1 : 0);
}

void launch_cg_p(cudaStream_t strm, const SmallCtx& c, int rp) {
  cg_p_kernel<<<counted(elem_grid(rp, rp)), NT, 0, strm>>>(c.st, rp, c.Ph, c.Rh, c.lds);
}

int launch_sylv_gemm(cudaStream_t strm, const SmallCtx& c, int r, const double* Z, double* Out, bool omega) {
  const int rp = r + c.s;
  const dim3 gg((rp + GBM - 1) / GBM, (rp + GBM - 1) / GBM);
  if (c.oz_scratch != nullptr && r >= c.oz_min_r)
    return launch_sylv_gemm_ozaki(strm, c.st, r, c.s, c.H, c.G, c.ldh, Z, Out, c.lds, omega, c.oz_scratch);
  if (c.df_small) {
    dfp* Hs = (dfp*)c.Hs;
    dfp* Gs = (dfp*)c.Gs;
    dfp* Zs = (dfp*)c.Zs;
    // columns of H and G are final once written: split only those added since the last call
    int launched = 2;
    if (*c.split_cols < r) {
      const int c0 = *c.split_cols;
      const int64_t E = (int64_t)rp * (r - c0);
      split_cols_kernel<<<counted((unsigned)((E + NT - 1) / NT)), NT, 0, strm>>>(c.st, rp, c0, r, c.H, c.ldh, Hs);
      launched += 1;
      if (c.G != c.H) {
        split_cols_kernel<<<counted((unsigned)((E + NT - 1) / NT)), NT, 0, strm>>>(c.st, rp, c0, r, c.G, c.ldh, Gs);
        launched += 1;
      }
      *c.split_cols = r;
    }
    const int64_t EZ = (int64_t)r * r;
    split_cols_kernel<<<counted((unsigned)((EZ + NT - 1) / NT)), NT, 0, strm>>>(c.st, r, 0, r, Z, c.lds, Zs);
    if (omega)
      sylv_gemm_df_kernel<true><<<counted(gg), NT, 0, strm>>>(c.st, r, c.s, Hs, Gs, c.ldh, Zs, Z, Out, c.lds, c.partials);
    else
      sylv_gemm_df_kernel<false><<<counted(gg), NT, 0, strm>>>(c.st, r, c.s, Hs, Gs, c.ldh, Zs, Z, Out, c.lds, nullptr);
    return launched;
  }
  if (omega)
    sylv_gemm_kernel<true><<<counted(gg), NT, 0, strm>>>(c.st, r, c.s, c.H, c.G, c.ldh, Z, Out, c.lds, c.partials);
  else
    sylv_gemm_kernel<false><<<counted(gg), NT, 0, strm>>>(c.st, r, c.s, c.H, c.G, c.ldh, Z, Out, c.lds, nullptr);
  return 1;
}

double sylv_gemm_flops(int r, int s) {
  // structural flops of [H Z, 0] + [Z G^T; 0] with block upper Hessenberg H, G
  double f = 0.0;
  const int rp = r + s;
  for (int a = 0; a < rp; ++a) {
    const int lo = std::max(0, (a / s - 1) * s);
    f += 2.0 * (double)r * (double)std::max(0, r - lo);  // row a of H Z (r columns) / column a of Z G^T
  }
  return 2.0 * f;
}

void launch_bicg_alpha(cudaStream_t strm, const SmallCtx& c) {
  bicg_alpha_kernel<<<counted(1), 32, 0, strm>>>(c.st, c.s, c.Rt, c.Qh, c.lds);
}

void launch_bicg_s(cudaStream_t strm, const SmallCtx& c, int rp) {
  bicg_s_kernel<<<counted(elem_grid(rp, rp)), NT, 0, strm>>>(c.st, rp, c.Sh, c.Rh, c.Qh, c.lds);
}

void launch_bicg_update(cudaStream_t strm, const SmallCtx& c, int k, int rp, int rpp) {
  bicg_update_kernel<<<counted(elem_grid(rpp, rpp)), NT, 0, strm>>>(c.st, c.hist, k, rp, rpp, c.s, c.Xh, c.Rh, c.Ph, c.Sh,
                                                           c.Th, c.Rt, c.lds, c.partials);
}

void launch_bicg_p(cudaStream_t strm, const SmallCtx& c, int rpp) {
  bicg_p_kernel<<<counted(elem_grid(rpp, rpp)), NT, 0, strm>>>(c.st, rpp, c.Ph, c.Rh, c.Qh, c.lds);
}

}  // namespace sylv
