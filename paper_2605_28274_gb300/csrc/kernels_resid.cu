// Float64 tall-skinny products for the true residual R = C1 C2^T - A X - X B of a
// factored iterate X = sum_i V_i X^_i W_i^T (the residual the convergence test
// of Algorithms 4.1/4.2 stands in for, eq. 3.6), and for the outer refinement of
// the mixed-precision mode.
//
// R is only ever applied to thin blocks (k <= 16 columns): R Omega and R^T Q.
// Those products cancel to ~1e-8 of their terms near convergence, so the tall
// products with the basis (tsg, tsu) accumulate in double-float arithmetic on
// the FP32 pipes: each float64 operand is split into hi + lo floats, products
// are formed with the error-free FMA product, sums with the error-free two-sum
// (Dekker 1971; Knuth TAOCP vol. 2), giving a unit roundoff of about 2^-48 at a
// fraction of the cost of float64 FMAs on this GPU (whose FP64 rate is 1/64 of
// its FP32 rate).  All explicit-rounding intrinsics, so nothing is contracted.
// Blocks of k vectors are n x k row-major.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace sylv {

namespace {

constexpr int TS_ROWS = 64;   // rows of Y staged in shared memory per tile
constexpr int TS_COLS = NT;   // basis columns per CTA (one per thread)

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl split(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ dfl split(float x) { return {x, 0.0f}; }

// acc += u * y for double-float u, y (the lo * lo term, ~2^-48 relative, is dropped), in the
// accumulation of Ogita, Rump, Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput.
// 26, 2005): the high word takes the rounded sum, the low word collects the exact two-sum
// error and the product's error; df_renorm folds the low word back every few terms, which
// keeps it a small correction (11 FP32 instructions per term instead of 14).
__device__ __forceinline__ void df_acc(dfl& acc, float ph, float pl) {
  const float s = __fadd_rn(acc.hi, ph);  // two-sum of acc.hi + ph
  const float bb = __fsub_rn(s, acc.hi);
  const float e = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(ph, bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pl));
}
__device__ __forceinline__ void df_renorm(dfl& acc) {
  const float s = __fadd_rn(acc.hi, acc.lo);
  acc.lo = __fsub_rn(acc.lo, __fsub_rn(s, acc.hi));
  acc.hi = s;
}
__device__ __forceinline__ void df_fma(dfl& acc, dfl u, dfl y) {
  const float ph = __fmul_rn(u.hi, y.hi);
  float pl = __fmaf_rn(u.hi, y.hi, -ph);  // exact error of the product
  pl = __fmaf_rn(u.hi, y.lo, pl);
  pl = __fmaf_rn(u.lo, y.hi, pl);
  df_acc(acc, ph, pl);
}
// a float u is exact in one word: no u.lo term
__device__ __forceinline__ void df_fma(dfl& acc, float u, dfl y) {
  const float ph = __fmul_rn(u, y.hi);
  float pl = __fmaf_rn(u, y.hi, -ph);
  pl = __fmaf_rn(u, y.lo, pl);
  df_acc(acc, ph, pl);
}
constexpr int DF_RENORM_EVERY = 8;  // terms between renormalisations of an accumulator

__device__ __forceinline__ dfl load_df(const double* p) { return split(*p); }
__device__ __forceinline__ float load_df(const float* p) { return *p; }

__device__ __forceinline__ double to_double(dfl a) { return (double)a.hi + (double)a.lo; }

// partial[rc][col][t] = sum over the rows of row-chunk rc of U[col][row] * Y[row][t]
// U: nb blocks of width su (block-row-major, element TU), Y: n x k row-major float64.
// A CTA covers cw columns (a power of two); with cw < NT its NT / cw thread slots split
// the rows of each tile (row i goes to slot i mod nslot) and are summed in slot order.
template <typename TU>
__global__ void __launch_bounds__(NT) tsg_kernel(int64_t n, int64_t rpc, const TU* __restrict__ U, int64_t bstride,
                                                 int su, int ncol, const double* __restrict__ Y, int k, int cw,
                                                 double* __restrict__ partial) {
  __shared__ dfl ys[TS_ROWS * 16];
  __shared__ double red[NT * 16];
  const int nslot = NT / cw, cl = threadIdx.x % cw, slot = threadIdx.x / cw;
  const int col = blockIdx.y * cw + cl;
  const int64_t r0 = (int64_t)blockIdx.x * rpc, r1 = min(n, r0 + rpc);
  dfl acc[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) acc[t] = {0.0f, 0.0f};
  const bool active = col < ncol;
  const int b = active ? col / su : 0, u = active ? col - b * su : 0;
  const TU* Ub = U + (int64_t)b * bstride + u;
  int terms = 0;
  for (int64_t base = r0; base < r1; base += TS_ROWS) {
    const int rows = (int)((r1 - base) < TS_ROWS ? (r1 - base) : TS_ROWS);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * k; e += NT) ys[e] = split(Y[base * k + e]);
    __syncthreads();
    if (active) {
      int i = slot;
      // four rows' loads in flight before their products
      for (; i + 3 * nslot < rows; i += 4 * nslot) {
        const auto u0 = load_df(Ub + (base + i) * su);
        const auto u1 = load_df(Ub + (base + i + nslot) * su);
        const auto u2 = load_df(Ub + (base + i + 2 * nslot) * su);
        const auto u3 = load_df(Ub + (base + i + 3 * nslot) * su);
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (t < k) {
            df_fma(acc[t], u0, ys[i * k + t]);
            df_fma(acc[t], u1, ys[(i + nslot) * k + t]);
            df_fma(acc[t], u2, ys[(i + 2 * nslot) * k + t]);
            df_fma(acc[t], u3, ys[(i + 3 * nslot) * k + t]);
          }
        terms += 4;
        if (terms >= DF_RENORM_EVERY) {
          terms = 0;
#pragma unroll
          for (int t = 0; t < 16; ++t) df_renorm(acc[t]);
        }
      }
      for (; i < rows; i += nslot) {
        const auto uv = load_df(Ub + (base + i) * su);
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (t < k) df_fma(acc[t], uv, ys[i * k + t]);
        if (++terms >= DF_RENORM_EVERY) {
          terms = 0;
#pragma unroll
          for (int t = 0; t < 16; ++t) df_renorm(acc[t]);
        }
      }
    }
  }
  if (nslot == 1) {
    if (active) {
      double* out = partial + ((int64_t)blockIdx.x * ncol + col) * k;
#pragma unroll
      for (int t = 0; t < 16; ++t)
        if (t < k) out[t] = to_double(acc[t]);
    }
    return;
  }
#pragma unroll
  for (int t = 0; t < 16; ++t) red[threadIdx.x * 16 + t] = to_double(acc[t]);
  __syncthreads();
  if (slot == 0 && active) {
    double* out = partial + ((int64_t)blockIdx.x * ncol + col) * k;
    for (int t = 0; t < k; ++t) {
      double v = 0.0;
      for (int q = 0; q < nslot; ++q) v += red[(q * cw + cl) * 16 + t];
      out[t] = v;
    }
  }
}

__global__ void tsg_reduce_kernel(const double* __restrict__ partial, int nrc, int64_t E, double* __restrict__ P) {
  const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (e >= E) return;
  double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;  // independent loads in flight, fixed order
  int c = 0;
  for (; c + 3 < nrc; c += 4) {
    v0 += partial[(int64_t)c * E + e];
    v1 += partial[(int64_t)(c + 1) * E + e];
    v2 += partial[(int64_t)(c + 2) * E + e];
    v3 += partial[(int64_t)(c + 3) * E + e];
  }
  for (; c < nrc; ++c) v0 += partial[(int64_t)c * E + e];
  P[e] = (v0 + v1) + (v2 + v3);
}

// Z[row][t] = beta * Z[row][t] + alpha * sum_col U[col][row] M[col][t]   (M: ncol x k row-major)
template <typename TU>
__global__ void __launch_bounds__(NT) tsu_kernel(int64_t n, const TU* __restrict__ U, int64_t bstride, int su,
                                                 int ncol, const double* __restrict__ M, int k, double alpha,
                                                 double beta, double* __restrict__ Z) {
  __shared__ dfl ms[64 * 16];
  const int64_t row = (int64_t)blockIdx.x * NT + threadIdx.x;
  dfl acc[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) acc[t] = {0.0f, 0.0f};
  for (int c0 = 0; c0 < ncol; c0 += 64) {
    const int cc = min(64, ncol - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < cc * k; e += NT) ms[e] = split(M[(int64_t)c0 * k + e]);
    __syncthreads();
    if (row < n) {
      int b = c0 / su, u = c0 - b * su;  // (block, column) of column c0 + c, advanced incrementally
      const TU* Ur = U + row * su;
      int c = 0;
      for (; c + 3 < cc; c += 4) {  // four columns' loads in flight before their products
        TU x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          x[q] = Ur[(int64_t)b * bstride + u];
          if (++u == su) {
            u = 0;
            ++b;
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const auto uv = load_df(&x[q]);
#pragma unroll
          for (int t = 0; t < 16; ++t)
            if (t < k) df_fma(acc[t], uv, ms[(c + q) * k + t]);
        }
        if ((c & (DF_RENORM_EVERY - 1)) == DF_RENORM_EVERY - 4) {
#pragma unroll
          for (int t = 0; t < 16; ++t) df_renorm(acc[t]);
        }
      }
      for (; c < cc; ++c) {
        const auto uv = load_df(Ur + (int64_t)b * bstride + u);
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (t < k) df_fma(acc[t], uv, ms[c * k + t]);
        if (++u == su) {
          u = 0;
          ++b;
        }
      }
    }
  }
  if (row < n) {
#pragma unroll
    for (int t = 0; t < 16; ++t)
      if (t < k) {
        double* z = Z + row * k + t;
        *z = (beta == 0.0 ? 0.0 : beta * *z) + alpha * to_double(acc[t]);
      }
  }
}

// out (r x k, row-major) = op(Xh) * in (r x k row-major), op = identity or transpose; Xh ld lds.
// A CTA owns 16 output rows x 16 columns; tiles of op(Xh) (16 x 64) and of in (64 x 16)
// are staged in shared memory, so the dependent chain per output runs on shared loads.
__global__ void __launch_bounds__(NT) small_apply_kernel(int r, int k, const double* __restrict__ Xh, int64_t lds,
                                                         int trans, const double* __restrict__ in,
                                                         double* __restrict__ out) {
  __shared__ double xs[16][65];
  __shared__ double is[64][17];
  const int ti = threadIdx.x >> 4, tt = threadIdx.x & 15;
  const int i0 = blockIdx.x * 16;
  const int i = i0 + ti;
  double acc = 0.0;
  for (int c0 = 0; c0 < r; c0 += 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * 64; e += NT) {
      int a, cc;
      if (!trans) {  // Xh[i + c*lds]: contiguous in i
        a = e % 16;
        cc = e / 16;
      } else {       // Xh[c + i*lds]: contiguous in c
        cc = e % 64;
        a = e / 64;
      }
      const int ii = i0 + a, c = c0 + cc;
      double x = 0.0;
      if (ii < r && c < r) x = trans ? Xh[c + (int64_t)ii * lds] : Xh[ii + (int64_t)c * lds];
      xs[a][cc] = x;
    }
    for (int e = threadIdx.x; e < 64 * 16; e += NT) {
      const int cc = e / 16, t = e % 16, c = c0 + cc;
      is[cc][t] = (c < r && t < k) ? in[(int64_t)c * k + t] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int cc = 0; cc < 64; ++cc) acc += xs[ti][cc] * is[cc][tt];
  }
  if (i < r && tt < k) out[(int64_t)i * k + tt] = acc;
}

// Y (n x k row-major) = alpha * Y + C (n x s row-major) * G (s x k row-major)
__global__ void lowrank_axpy_kernel(int64_t n, int s, int k, const double* __restrict__ C,
                                    const double* __restrict__ G, double alpha, double* __restrict__ Y) {
  const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (e >= n * k) return;
  const int64_t row = e / k;
  const int t = (int)(e - row * k);
  double acc = 0.0;
  for (int c = 0; c < s; ++c) acc += C[row * s + c] * G[c * k + t];
  Y[e] = alpha * Y[e] + acc;
}

// out (rows x 16) = [a | b] with a, b rows x 8 (all row-major)
__global__ void interleave_kernel(int64_t rows, const double* __restrict__ a, const double* __restrict__ b,
                                  double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (e >= rows * 16) return;
  const int64_t r = e >> 4;
  const int c = (int)(e & 15);
  out[e] = c < 8 ? a[r * 8 + c] : b[r * 8 + c - 8];
}

// a, b (rows x 8) = columns 0..7 and 8..15 of in (rows x 16)
__global__ void deinterleave_kernel(int64_t rows, const double* __restrict__ in, double* __restrict__ a,
                                    double* __restrict__ b) {
  const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (e >= rows * 16) return;
  const int64_t r = e >> 4;
  const int c = (int)(e & 15);
  if (c < 8) a[r * 8 + c] = in[e];
  else b[r * 8 + c - 8] = in[e];
}

// y += a * x, element-wise
__global__ void axpy_kernel(int64_t count, double a, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (e < count) y[e] += a * x[e];
}

// out = -(X1 + X2), element-wise
__global__ void neg_sum_kernel(int64_t count, const double* __restrict__ X1, const double* __restrict__ X2,
                               double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (e < count) out[e] = -(X1[e] + X2[e]);
}

// sum of squares of x[0..count) -> partial per CTA (deterministic), then out[0] by the last CTA
__global__ void sumsq_kernel(int64_t count, const double* __restrict__ x, double* __restrict__ partials,
                             unsigned int* ticket, double* __restrict__ out) {
  __shared__ double sh[32];
  __shared__ int last_sh;
  double v = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < count; i += (int64_t)gridDim.x * NT) v += x[i] * x[i];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = v;
  if (last_cta(ticket, &last_sh)) {
    const double t = cta_sum(partials, (int)gridDim.x, 1, 0, sh);
    if (threadIdx.x == 0) {
      *out = t;
    }
  }
}

// out = trace(G1 G2) for symmetric s x s G1, G2 (row-major): ||C1 C2^T||_F^2 from the two Grams.
__global__ void trace_prod_kernel(int s, const double* __restrict__ G1, const double* __restrict__ G2,
                                  double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) t += G1[i * s + j] * G2[j * s + i];
  *out = t;
}

}  // namespace

int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
}

int64_t tsg_partial_elems(int64_t ncol, int k) {
  return ((int64_t)4 * sm_count() + ncol / TS_COLS + 2) * TS_COLS * k;
}

template <typename TU>
void launch_tsg(cudaStream_t strm, int64_t n, const TU* U, int64_t bstride, int su, int nb, const double* Y, int k,
                double* partial, int max_rc, double* P) {
  const int ncol = nb * su;
  if (ncol == 0) return;
  // cw columns per CTA (narrow blocks: fewer columns, more row slots); about four CTAs
  // per SM over (row chunk, column chunk); at least 256 rows per chunk
  int cw = 1;
  while (cw < ncol && cw < TS_COLS) cw <<= 1;
  const int cchunks = (ncol + cw - 1) / cw;
  int rc = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256),
                                  std::max(1, (4 * sm_count() + cchunks - 1) / cchunks));
  if (max_rc > 0) rc = std::min(rc, max_rc);
  const int64_t rpc = (n + rc - 1) / rc;
  rc = (int)((n + rpc - 1) / rpc);
  const dim3 g((unsigned)rc, (unsigned)cchunks);
  tsg_kernel<TU><<<counted(g), NT, 0, strm>>>(n, rpc, U, bstride, su, ncol, Y, k, cw, partial);
  const int64_t E = (int64_t)ncol * k;
  tsg_reduce_kernel<<<counted((unsigned)((E + NT - 1) / NT)), NT, 0, strm>>>(partial, rc, E, P);
}

template <typename TU>
void launch_tsu(cudaStream_t strm, int64_t n, const TU* U, int64_t bstride, int su, int nb, const double* M, int k,
                double alpha, double beta, double* Z) {
  const int ncol = nb * su;  // ncol = 0: Z = beta Z
  if (n == 0) return;
  tsu_kernel<TU><<<counted((unsigned)((n + NT - 1) / NT)), NT, 0, strm>>>(n, U, bstride, su, ncol, M, k, alpha, beta, Z);
}

void launch_small_apply(cudaStream_t strm, int r, int k, const double* Xh, int64_t lds, bool trans, const double* in,
                        double* out) {
  if (r == 0 || k == 0) return;
  small_apply_kernel<<<counted((unsigned)((r + 15) / 16)), NT, 0, strm>>>(r, k, Xh, lds, trans ? 1 : 0, in, out);
}

void launch_lowrank_axpy(cudaStream_t strm, int64_t n, int s, int k, const double* C, const double* G, double alpha,
                         double* Y) {
  lowrank_axpy_kernel<<<counted((unsigned)((n * k + NT - 1) / NT)), NT, 0, strm>>>(n, s, k, C, G, alpha, Y);
}

void launch_interleave(cudaStream_t strm, int64_t rows, const double* a, const double* b, double* out) {
  if (rows == 0) return;
  interleave_kernel<<<counted((unsigned)((rows * 16 + NT - 1) / NT)), NT, 0, strm>>>(rows, a, b, out);
}

void launch_deinterleave(cudaStream_t strm, int64_t rows, const double* in, double* a, double* b) {
  if (rows == 0) return;
  deinterleave_kernel<<<counted((unsigned)((rows * 16 + NT - 1) / NT)), NT, 0, strm>>>(rows, in, a, b);
}

void launch_axpy(cudaStream_t strm, int64_t count, double a, const double* x, double* y) {
  if (count == 0) return;
  axpy_kernel<<<counted((unsigned)((count + NT - 1) / NT)), NT, 0, strm>>>(count, a, x, y);
}

void launch_neg_sum(cudaStream_t strm, int64_t count, const double* X1, const double* X2, double* out) {
  if (count == 0) return;
  neg_sum_kernel<<<counted((unsigned)((count + NT - 1) / NT)), NT, 0, strm>>>(count, X1, X2, out);
}

void launch_sumsq(cudaStream_t strm, int64_t count, const double* x, double* partials, unsigned int* ticket,
                  double* out) {
  const int grid = (int)std::min<int64_t>(256, std::max<int64_t>(1, (count + NT - 1) / NT));
  sumsq_kernel<<<counted(grid), NT, 0, strm>>>(count, x, partials, ticket, out);
}

void launch_trace_prod(cudaStream_t strm, int s, const double* G1, const double* G2, double* out) {
  trace_prod_kernel<<<counted(1), 32, 0, strm>>>(s, G1, G2, out);
}

template void launch_tsg<float>(cudaStream_t, int64_t, const float*, int64_t, int, int, const double*, int, double*,
                                int, double*);
template void launch_tsg<double>(cudaStream_t, int64_t, const double*, int64_t, int, int, const double*, int, double*,
                                 int, double*);
template void launch_tsu<float>(cudaStream_t, int64_t, const float*, int64_t, int, int, const double*, int, double,
                                double, double*);
template void launch_tsu<double>(cudaStream_t, int64_t, const double*, int64_t, int, int, const double*, int, double,
                                 double, double*);

// out[i] ~ N(0, 1), i < count: the SplitMix64 stream (Steele, Lea, Flood, OOPSLA 2014) from
// seed, whose output j is mix(seed + (j + 1) * 0x9E3779B97F4A7C15), taken in pairs (u1, u2) of
// 53-bit uniforms (u1 in (0, 1]) and Box-Muller: out[2i] = r cos(2 pi u2), out[2i+1] = r sin(2 pi u2),
// r = sqrt(-2 ln u1).  One thread per pair.
namespace {
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t j) {
  uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void __launch_bounds__(NT) gauss_probes_kernel(double* __restrict__ out, int64_t count, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (2 * i >= count) return;
  const double u1 = ((double)(splitmix64_at(seed, 2 * (uint64_t)i) >> 11) + 1.0) * 0x1.0p-53;
  const double u2 = (double)(splitmix64_at(seed, 2 * (uint64_t)i + 1) >> 11) * 0x1.0p-53;
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  out[2 * i] = r * cs;
  if (2 * i + 1 < count) out[2 * i + 1] = r * sn;
}
}  // namespace

void launch_gauss_probes(cudaStream_t strm, double* out, size_t count, uint64_t seed) {
  if (count == 0) return;
  const int64_t pairs = (int64_t)((count + 1) / 2);
  gauss_probes_kernel<<<counted((unsigned)((pairs + NT - 1) / NT)), NT, 0, strm>>>(out, (int64_t)count, seed);
}

}  // namespace sylv
