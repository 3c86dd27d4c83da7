// Device-side definitions shared by the solver kernels.
//
// The whole iteration of Algorithms 4.1/4.2 runs on the device: the scalars
// alpha, beta, omega, rho, the residual norm and the convergence flag live in
// a DevState in device memory.  Every kernel first reads DevState::status and
// returns at once when the solve has stopped (converged, breakdown, non-finite),
// so the host can enqueue iterations ahead of the device and poll only every
// few iterations.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sylv {

// ST_WAIT_TIMEOUT: a kernel's bounded wait on its own asynchronous copies or tensor-core
// operations gave up (the kernel returned without its result).
enum DevStatus : int { ST_RUNNING = 0, ST_CONVERGED = 1, ST_BREAKDOWN = 2, ST_NONFINITE = 3, ST_WAIT_TIMEOUT = 4 };

// Tickets for the "last CTA finishes the reduction" pattern, one per kernel kind.
enum Ticket : int {
  TK_CG_Q = 0,
  TK_CG_UPD = 1,
  TK_BI_T = 2,
  TK_BI_UPD = 3,
  TK_GP_ZETA = 4,
  TK_OB_H0 = 5,  // the H reduction + coefficient digits of basis side 0 / 1 (concurrent streams)
  TK_OB_H1 = 6,
  TK_NUM = 8
};

struct DevState {
  double rho, alpha, beta, omega;  // GPBiCG: omega holds zeta
  double eta;    // GPBiCG only
  double r0;     // ||R^_0||_F
  double rnorm;  // ||R^_k||_F of the latest iterate
  double tol;
  int status;    // DevStatus
  int iters;     // completed iterations
  int exhausted[2];  // per basis side: the block Krylov space is exhausted
  int breakdown_where;  // diagnostic code of the first breakdown
  int pad;
  unsigned int tickets[TK_NUM];
};

constexpr int NT = 256;  // threads per CTA for the streaming kernels

// The same answer in every thread of the CTA, which must all call it (every kernel does, as its
// first statement).  Kernels on the two basis streams run while the small side (or the other
// basis) writes the status word, so two threads of one CTA can read different values; a CTA
// split between "stopped" and "running" would run its cooperative parts (shared-memory staging,
// barriers, tensor-memory allocation, bulk copies issued by one thread) with threads missing.
__device__ __forceinline__ bool stopped(const DevState* st) {
  const bool mine = st != nullptr && *((volatile const int*)&st->status) != ST_RUNNING;
  return __syncthreads_or(mine ? 1 : 0) != 0;
}

// Deterministic block-wide sum of one double per thread (NT threads).
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    sh[0] = t;
  }
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

// Sum of partials[i * stride + off], i < nb, by every thread of the calling CTA: each thread
// adds a strided subset, then block_sum (a fixed order).  All threads of the CTA must call it.
// The last CTA of a reduction uses it: one thread adding thousands of partials in sequence
// spent tens of microseconds in float64 additions on this GPU.
__device__ __forceinline__ double cta_sum(const double* partials, int nb, int stride, int off, double* sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v += __ldcg(partials + (int64_t)i * stride + off);
  return block_sum(v, sh);
}

// Last-CTA detection after each CTA has written its partial result.
// Returns true in exactly one CTA (the last to arrive); that CTA resets the ticket.
__device__ __forceinline__ bool last_cta(unsigned int* ticket, int* flag_sh) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(ticket, 1u);
    *flag_sh = (t == gridDim.x * gridDim.y - 1) ? 1 : 0;
  }
  __syncthreads();
  const bool last = *flag_sh != 0;
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) *ticket = 0u;
  }
  return last;
}

// Cholesky G = R^T R of a symmetric s x s matrix (G[u*s+t], s <= 8) with upper R
// (column-major R[i + j*s]) and its inverse Ri.  A pivot <= thr is a failure
// (returns 1).  Single thread.
__device__ __forceinline__ int chol_small(const double* G, int s, double thr, double* R, double* Ri) {
  for (int e = 0; e < 64; ++e) {
    R[e] = 0.0;
    Ri[e] = 0.0;
  }
  for (int j = 0; j < s; ++j) {
    double d = G[j * s + j];
    for (int k = 0; k < j; ++k) d -= R[k + j * s] * R[k + j * s];
    if (!(d > thr)) return 1;
    const double rjj = sqrt(d);
    R[j + j * s] = rjj;
    for (int i = j + 1; i < s; ++i) {
      double g = G[j * s + i];
      for (int k = 0; k < j; ++k) g -= R[k + j * s] * R[k + i * s];
      R[j + i * s] = g / rjj;
    }
  }
  for (int j = 0; j < s; ++j) {
    Ri[j + j * s] = 1.0 / R[j + j * s];
    for (int i = j - 1; i >= 0; --i) {
      double acc = 0.0;
      for (int k = i; k < j; ++k) acc += Ri[i + k * s] * R[k + j * s];
      Ri[i + j * s] = -acc / R[j + j * s];
    }
  }
  return 0;
}

}  // namespace sylv
