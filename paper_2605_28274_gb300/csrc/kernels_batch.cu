// Batched factorized CG for many Lyapunov equations A_i X_i + X_i A_i^T = C_i C_i^T
// (Algorithm 4.1 with the one-basis, one-product form of Sec. 4.3) of uneven n_i
// and s_i, one persistent launch per phase for all instances.
//
// Row phases (sparse apply, Gram, update, scale) walk a fixed work list of
// (instance, row chunk) items; small-matrix phases walk every running
// instance's element tiles; per-instance phases (reductions, Cholesky, scalar
// updates) take one CTA or thread per instance.  Every kernel reads the
// instance's iteration index k and status from device memory, so the 15
// launches of one iteration are captured once as a CUDA graph and replayed;
// converged instances drop out of every phase.  All sums are taken in a fixed
// order (per-item / per-tile partials, added in index order): results do not
// depend on the schedule.
#include <cstring>

#include "common.cuh"
#include "kernels.h"

namespace sylv {

namespace {

constexpr int TE = 8;  // elements per thread per tile in the small phases

__device__ __forceinline__ bool running(const BatchInst& I) {
  return *((volatile const int*)&I.st->status) == ST_RUNNING;
}

template <int S>
__device__ __forceinline__ void ldv(const double* p, double (&v)[S]) {
  if constexpr (S % 2 == 0) {
#pragma unroll
    for (int i = 0; i < S / 2; ++i) {
      const double2 q = *(reinterpret_cast<const double2*>(p) + i);
      v[2 * i] = q.x;
      v[2 * i + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int u = 0; u < S; ++u) v[u] = p[u];
  }
}

template <int S>
__device__ __forceinline__ void stv(double* p, const double (&v)[S]) {
  if constexpr (S % 2 == 0) {
#pragma unroll
    for (int i = 0; i < S / 2; ++i) *(reinterpret_cast<double2*>(p) + i) = make_double2(v[2 * i], v[2 * i + 1]);
  } else {
#pragma unroll
    for (int u = 0; u < S; ++u) p[u] = v[u];
  }
}

// Block-wide sum of an S x S register tile into out[0..S*S) (all NT threads).
template <int S>
__device__ __forceinline__ void reduce_tile(double (&acc)[S][S], double* out, double* sh) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
#pragma unroll
  for (int u = 0; u < S; ++u)
#pragma unroll
    for (int t = 0; t < S; ++t) {
      double v = acc[u][t];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (l == 0) sh[w * S * S + u * S + t] = v;
    }
  __syncthreads();
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < NT / 32; ++i) s += sh[i * S * S + e];
    out[e] = s;
  }
}

#define BATCH_S_SWITCH(s, CALL) \
  switch (s) {                  \
    case 1: CALL(1); break;     \
    case 2: CALL(2); break;     \
    case 3: CALL(3); break;     \
    case 4: CALL(4); break;     \
    case 5: CALL(5); break;     \
    case 6: CALL(6); break;     \
    case 7: CALL(7); break;     \
    default: CALL(8); break;    \
  }

// ---------------------------------------------------------------- row phases
// Y = A V_q - V_{q-1} H_{q-1,q}   (block Lanczos three-term recurrence, q = k)
template <int S>
__device__ void ph_spmm(const BatchInst& I, int64_t r0, int64_t r1) {
  const int q = I.k;
  const int64_t bs = I.n * S;
  const double* Vq = I.V + q * bs;
  double* Y = I.V + (q + 1) * bs;
  const double* Vp = q > 0 ? I.V + (q - 1) * bs : nullptr;
  const double* M = q > 0 ? I.H + (int64_t)(q - 1) * S + (int64_t)q * S * I.ldh : nullptr;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    double y[S];
#pragma unroll
    for (int t = 0; t < S; ++t) y[t] = 0.0;
    const int p0 = __ldg(I.rp + row), p1 = __ldg(I.rp + row + 1);
    for (int p = p0; p < p1; ++p) {
      const double v = __ldg(I.val + p);
      double x[S];
      ldv<S>(Vq + (int64_t)__ldg(I.ci + p) * S, x);
#pragma unroll
      for (int t = 0; t < S; ++t) y[t] += v * x[t];
    }
    if (Vp) {
      double xp[S];
      ldv<S>(Vp + row * S, xp);
#pragma unroll
      for (int t = 0; t < S; ++t)
#pragma unroll
        for (int u = 0; u < S; ++u) y[t] -= xp[u] * M[u + (int64_t)t * I.ldh];
    }
    stv<S>(Y + row * S, y);
  }
}

// partial = V_q^T Y over the chunk's rows
template <int S>
__device__ void ph_gram(const BatchInst& I, int64_t r0, int64_t r1, double* out, double* sh) {
  const int q = I.k;
  const int64_t bs = I.n * S;
  const double* Vq = I.V + q * bs;
  const double* Y = Vq + bs;
  double acc[S][S];
#pragma unroll
  for (int u = 0; u < S; ++u)
#pragma unroll
    for (int t = 0; t < S; ++t) acc[u][t] = 0.0;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    double v[S], y[S];
    ldv<S>(Vq + row * S, v);
    ldv<S>(Y + row * S, y);
#pragma unroll
    for (int u = 0; u < S; ++u)
#pragma unroll
      for (int t = 0; t < S; ++t) acc[u][t] += v[u] * y[t];
  }
  reduce_tile<S>(acc, out, sh);
}

// Y -= V_q H_{q,q}; partial = Y^T Y
template <int S>
__device__ void ph_update(const BatchInst& I, int64_t r0, int64_t r1, double* out, double* sh) {
  const int q = I.k;
  const int64_t bs = I.n * S;
  const double* Vq = I.V + q * bs;
  double* Y = I.V + (q + 1) * bs;
  const double* Hq = I.H + (int64_t)q * S + (int64_t)q * S * I.ldh;
  double acc[S][S];
#pragma unroll
  for (int u = 0; u < S; ++u)
#pragma unroll
    for (int t = 0; t < S; ++t) acc[u][t] = 0.0;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    double v[S], y[S];
    ldv<S>(Vq + row * S, v);
    ldv<S>(Y + row * S, y);
#pragma unroll
    for (int t = 0; t < S; ++t)
#pragma unroll
      for (int u = 0; u < S; ++u) y[t] -= v[u] * Hq[u + (int64_t)t * I.ldh];
    stv<S>(Y + row * S, y);
#pragma unroll
    for (int u = 0; u < S; ++u)
#pragma unroll
      for (int t = 0; t < S; ++t) acc[u][t] += y[u] * y[t];
  }
  reduce_tile<S>(acc, out, sh);
}

// Y <- Y Rinv (upper triangular); with out != NULL also partial = Y^T Y
template <int S>
__device__ void ph_scale(const BatchInst& I, int64_t r0, int64_t r1, double* out, double* sh) {
  const int q = I.k;
  const int64_t bs = I.n * S;
  double* Y = I.V + (q + 1) * bs;
  double ri[S * S];
#pragma unroll
  for (int e = 0; e < S * S; ++e) ri[e] = I.Rinv[e];
  double acc[S][S];
#pragma unroll
  for (int u = 0; u < S; ++u)
#pragma unroll
    for (int t = 0; t < S; ++t) acc[u][t] = 0.0;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    double y[S], z[S];
    ldv<S>(Y + row * S, y);
#pragma unroll
    for (int t = 0; t < S; ++t) {
      double a = 0.0;
#pragma unroll
      for (int u = 0; u <= t; ++u) a += y[u] * ri[u + t * S];
      z[t] = a;
    }
    stv<S>(Y + row * S, z);
#pragma unroll
    for (int u = 0; u < S; ++u)
#pragma unroll
      for (int t = 0; t < S; ++t) acc[u][t] += z[u] * z[t];
  }
  if (out) reduce_tile<S>(acc, out, sh);
}

enum RowPhase { RP_SPMM = 0, RP_GRAM = 1, RP_UPDATE = 2, RP_SCALE_SELF = 3, RP_SCALE = 4 };

template <int PH>
__global__ void __launch_bounds__(NT) k_rows(BatchCtx c) {
  __shared__ double sh[(NT / 32) * 64];
  for (int it = blockIdx.x; it < c.nitems; it += gridDim.x) {
    const int2 w = c.items[it];
    const BatchInst& I = c.insts[w.x];
    if (!running(I)) continue;  // uniform over the CTA
    const int64_t r0 = w.y, r1 = min(I.n, r0 + (int64_t)c.chunk);
    double* gout = c.gpart + (int64_t)it * 64;
    double* sout = c.spart + (int64_t)it * 64;
    if (PH == RP_SPMM) {
#define CALL(SV) ph_spmm<SV>(I, r0, r1)
      BATCH_S_SWITCH(I.s, CALL)
#undef CALL
    } else if (PH == RP_GRAM) {
#define CALL(SV) ph_gram<SV>(I, r0, r1, gout, sh)
      BATCH_S_SWITCH(I.s, CALL)
#undef CALL
    } else if (PH == RP_UPDATE) {
#define CALL(SV) ph_update<SV>(I, r0, r1, sout, sh)
      BATCH_S_SWITCH(I.s, CALL)
#undef CALL
    } else if (PH == RP_SCALE_SELF) {
#define CALL(SV) ph_scale<SV>(I, r0, r1, sout, sh)
      BATCH_S_SWITCH(I.s, CALL)
#undef CALL
    } else {
#define CALL(SV) ph_scale<SV>(I, r0, r1, nullptr, sh)
      BATCH_S_SWITCH(I.s, CALL)
#undef CALL
    }
  }
}

// ---------------------------------------------------------------- per-instance phases
// H_{q,q} = sum of the Gram partials of the instance's items (fixed order)
__global__ void __launch_bounds__(64) k_reduce_h(BatchCtx c) {
  for (int i = blockIdx.x; i < c.count; i += gridDim.x) {
    const BatchInst& I = c.insts[i];
    if (!running(I)) continue;
    const int s = I.s, q = I.k;
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
      double v = 0.0;
      for (int it = I.item_begin; it < I.item_end; ++it) v += c.gpart[(int64_t)it * 64 + e];
      const int u = e / s, t = e - u * s;
      I.H[(int64_t)q * s + u + ((int64_t)q * s + t) * I.ldh] = v;
    }
  }
}

// CholQR pass on the reduced self-Gram (see the single-instance chol kernel for the
// exhaustion / rank-loss readings).  Pass 2 writes H_{q+1,q} = R2 R1 and H_{q,q+1}.
__global__ void __launch_bounds__(64) k_chol(BatchCtx c, int pass) {
  __shared__ double G[64], R[64], Ri[64];
  for (int i = blockIdx.x; i < c.count; i += gridDim.x) {
    BatchInst& I = c.insts[i];
    if (!running(I)) continue;
    const int s = I.s, q = I.k, E = s * s;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
      double v = 0.0;
      for (int it = I.item_begin; it < I.item_end; ++it) v += c.spart[(int64_t)it * 64 + e];
      G[e] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      DevState* st = I.st;
      bool finite = true;
      double tr = 0.0;
      for (int e = 0; e < E; ++e) finite = finite && isfinite(G[e]);
      for (int u = 0; u < s; ++u) tr += G[u * s + u];
      int exh = st->exhausted[0];
      int bad = 0;
      if (pass == 1) {
        double hsq = 0.0;  // ||H_{1:q+1,q}||^2: blocks q-1 and q of column block q
        const int64_t rlo = q > 0 ? (int64_t)(q - 1) * s : 0, rhi = (int64_t)(q + 1) * s;
        for (int t = 0; t < s; ++t)
          for (int64_t rr = rlo; rr < rhi; ++rr) {
            const double h = I.H[rr + ((int64_t)q * s + t) * I.ldh];
            hsq += h * h;
          }
        const double nu2 = hsq + tr;
        if (!finite) {
          st->status = ST_NONFINITE;
          st->breakdown_where = 100;
          bad = 1;
        } else if (!exh && tr <= c.delta * c.delta * nu2) {
          exh = 1;
          st->exhausted[0] = 1;
        }
        if (!bad && !exh && chol_small(G, s, c.delta * c.delta * nu2, R, Ri)) {
          st->status = ST_BREAKDOWN;
          st->breakdown_where = 10;
          bad = 1;
        }
      } else if (!exh) {
        if (!finite || chol_small(G, s, 0.0, R, Ri)) {
          st->status = finite ? ST_BREAKDOWN : ST_NONFINITE;
          st->breakdown_where = 11;
          bad = 1;
        }
      }
      if (!bad) {
        if (exh)
          for (int e = 0; e < 64; ++e) R[e] = Ri[e] = 0.0;
        for (int e = 0; e < E; ++e) I.Rinv[e] = Ri[e];
        if (pass == 1) {
          for (int e = 0; e < E; ++e) I.R1[e] = R[e];
        } else {
          for (int jj = 0; jj < s; ++jj)
            for (int ii = 0; ii < s; ++ii) {
              double acc = 0.0;
              for (int kk = 0; kk < s; ++kk) acc += R[ii + kk * s] * I.R1[kk + jj * s];
              if (exh) acc = 0.0;
              I.H[(int64_t)(q + 1) * s + ii + ((int64_t)q * s + jj) * I.ldh] = acc;      // H_{q+1,q}
              I.H[(int64_t)q * s + jj + ((int64_t)(q + 1) * s + ii) * I.ldh] = acc;      // H_{q,q+1}
            }
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- small-matrix phases (Sec. 4.3)
// M = [H P^, 0]  (block tridiagonal H: three s-blocks per row)
__global__ void __launch_bounds__(NT) k_lyap_m(BatchCtx c) {
  for (int i = 0; i < c.count; ++i) {
    const BatchInst& I = c.insts[i];
    if (!running(I)) continue;
    const int s = I.s, r = (I.k + 1) * s, rp = r + s;
    const int64_t E = (int64_t)rp * rp, per = (int64_t)NT * TE;
    const int ntiles = (int)((E + per - 1) / per);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
      for (int j = 0; j < TE; ++j) {
        const int64_t e = tile * per + (int64_t)j * NT + threadIdx.x;
        if (e >= E) break;
        const int a = (int)(e % rp), b = (int)(e / rp);
        double m = 0.0;
        if (b < r) {
          const int ba = a / s;
          const int c0 = max(0, (ba - 1) * s), c1 = min(r, (ba + 2) * s);
          for (int cc = c0; cc < c1; ++cc) m += I.H[a + (int64_t)cc * I.ldh] * I.P[cc + (int64_t)b * I.lds];
        }
        I.M[a + (int64_t)b * I.lds] = m;
      }
  }
}

// Q^ = M + M^T; per-tile partial of <P^, Q^(1:r,1:r)>
__global__ void __launch_bounds__(NT) k_lyap_q(BatchCtx c) {
  __shared__ double sh[32];
  for (int i = 0; i < c.count; ++i) {
    const BatchInst& I = c.insts[i];
    if (!running(I)) continue;
    const int s = I.s, r = (I.k + 1) * s, rp = r + s;
    const int64_t E = (int64_t)rp * rp, per = (int64_t)NT * TE;
    const int ntiles = (int)((E + per - 1) / per);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      double pq = 0.0;
      for (int j = 0; j < TE; ++j) {
        const int64_t e = tile * per + (int64_t)j * NT + threadIdx.x;
        if (e >= E) break;
        const int a = (int)(e % rp), b = (int)(e / rp);
        const double qv = I.M[a + (int64_t)b * I.lds] + I.M[b + (int64_t)a * I.lds];
        I.Q[a + (int64_t)b * I.lds] = qv;
        if (a < r && b < r) pq += I.P[a + (int64_t)b * I.lds] * qv;
      }
      pq = block_sum(pq, sh);
      if (threadIdx.x == 0) I.psm[tile] = pq;
    }
  }
}

// X^ += alpha P^ (extent r), R^ -= alpha Q^ (extent r+s); per-tile partial of ||R^||^2
__global__ void __launch_bounds__(NT) k_cg_update(BatchCtx c) {
  __shared__ double sh[32];
  for (int i = 0; i < c.count; ++i) {
    const BatchInst& I = c.insts[i];
    if (!running(I)) continue;
    const int s = I.s, r = (I.k + 1) * s, rp = r + s;
    const double alpha = I.st->alpha;
    const int64_t E = (int64_t)rp * rp, per = (int64_t)NT * TE;
    const int ntiles = (int)((E + per - 1) / per);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      double rr = 0.0;
      for (int j = 0; j < TE; ++j) {
        const int64_t e = tile * per + (int64_t)j * NT + threadIdx.x;
        if (e >= E) break;
        const int a = (int)(e % rp), b = (int)(e / rp);
        const int64_t x = a + (int64_t)b * I.lds;
        if (a < r && b < r) I.X[x] = I.X[x] + alpha * I.P[x];
        const double v = I.R[x] - alpha * I.Q[x];
        I.R[x] = v;
        rr += v * v;
      }
      rr = block_sum(rr, sh);
      if (threadIdx.x == 0) I.psm[tile] = rr;
    }
  }
}

// P^ = R^ + beta P^ (extent r+s)
__global__ void __launch_bounds__(NT) k_cg_p(BatchCtx c) {
  for (int i = 0; i < c.count; ++i) {
    const BatchInst& I = c.insts[i];
    if (!running(I)) continue;
    const int s = I.s, rp = (I.k + 2) * s;
    const double beta = I.st->beta;
    const int64_t E = (int64_t)rp * rp, per = (int64_t)NT * TE;
    const int ntiles = (int)((E + per - 1) / per);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
      for (int j = 0; j < TE; ++j) {
        const int64_t e = tile * per + (int64_t)j * NT + threadIdx.x;
        if (e >= E) break;
        const int a = (int)(e % rp), b = (int)(e / rp);
        const int64_t x = a + (int64_t)b * I.lds;
        I.P[x] = I.R[x] + beta * I.P[x];
      }
  }
}

// alpha = rho / <P^, Q^(1:r,1:r)>  (one thread per instance, tiles added in order)
__global__ void k_alpha(BatchCtx c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.count) return;
  const BatchInst& I = c.insts[i];
  if (!running(I)) return;
  const int rp = (I.k + 2) * I.s;
  const int64_t per = (int64_t)NT * TE;
  const int ntiles = (int)(((int64_t)rp * rp + per - 1) / per);
  double tot = 0.0;
  for (int t = 0; t < ntiles; ++t) tot += I.psm[t];
  DevState* st = I.st;
  if (!isfinite(tot)) {
    st->status = ST_NONFINITE;
    st->breakdown_where = 1;
  } else if (!(tot > 0.0)) {
    st->status = ST_BREAKDOWN;
    st->breakdown_where = 2;
  } else {
    st->alpha = st->rho / tot;
  }
}

// residual norm, history, convergence test, rho, beta (one thread per instance)
__global__ void k_test(BatchCtx c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.count) return;
  const BatchInst& I = c.insts[i];
  if (!running(I)) return;
  const int k = I.k, rp = (k + 2) * I.s;
  const int64_t per = (int64_t)NT * TE;
  const int ntiles = (int)(((int64_t)rp * rp + per - 1) / per);
  double tot = 0.0;
  for (int t = 0; t < ntiles; ++t) tot += I.psm[t];
  DevState* st = I.st;
  const double rn = sqrt(tot);
  I.hist[k + 1] = rn / st->r0;
  st->rnorm = rn;
  st->iters = k + 1;
  if (!isfinite(rn)) {
    st->status = ST_NONFINITE;
    st->breakdown_where = 3;
  } else if (rn <= st->r0 * st->tol) {
    st->status = ST_CONVERGED;
  } else {
    st->beta = tot / st->rho;
    st->rho = tot;
  }
}

// advance k of the running instances and count them (one thread)
__global__ void k_advance(BatchCtx c) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int run = 0;
  for (int i = 0; i < c.count; ++i) {
    BatchInst& I = c.insts[i];
    if (I.st->status == ST_RUNNING) {
      I.k += 1;
      ++run;
    }
  }
  *c.running = run;
}

}  // namespace

void launch_batch_spmm_gram(cudaStream_t st, const BatchCtx& c) {
  k_rows<RP_SPMM><<<counted(c.grid), NT, 0, st>>>(c);
  k_rows<RP_GRAM><<<counted(c.grid), NT, 0, st>>>(c);
}

void launch_batch_iteration(cudaStream_t st, const BatchCtx& c) {
  const int gi = (c.count + 63) / 64;
  const int gs = c.sgrid;
  k_rows<RP_SPMM><<<counted(c.grid), NT, 0, st>>>(c);
  k_rows<RP_GRAM><<<counted(c.grid), NT, 0, st>>>(c);
  k_reduce_h<<<counted(c.count), 64, 0, st>>>(c);
  k_rows<RP_UPDATE><<<counted(c.grid), NT, 0, st>>>(c);
  k_chol<<<counted(c.count), 64, 0, st>>>(c, 1);
  k_rows<RP_SCALE_SELF><<<counted(c.grid), NT, 0, st>>>(c);
  k_chol<<<counted(c.count), 64, 0, st>>>(c, 2);
  k_rows<RP_SCALE><<<counted(c.grid), NT, 0, st>>>(c);
  k_lyap_m<<<counted(gs), NT, 0, st>>>(c);
  k_lyap_q<<<counted(gs), NT, 0, st>>>(c);
  k_alpha<<<counted(gi), 64, 0, st>>>(c);
  k_cg_update<<<counted(gs), NT, 0, st>>>(c);
  k_test<<<counted(gi), 64, 0, st>>>(c);
  k_cg_p<<<counted(gs), NT, 0, st>>>(c);
  k_advance<<<counted(1), 32, 0, st>>>(c);
}

}  // namespace sylv
