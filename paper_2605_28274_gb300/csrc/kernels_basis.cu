// Basis-side kernels of the factorized Krylov methods: the sparse apply and the
// block orthogonalisation that realise A V_k = V_{k+1} H_{k+1,k} (eq. 3.4) for
// block Lanczos (Algorithm 4.1) and block Arnoldi (Algorithm 4.2).
//
// Data layout: a basis block V_b (n x s) is stored row-major, so one row's s
// coefficients are contiguous (one 16/32-byte vector) and consecutive rows are
// consecutive in memory.  The sparse apply gathers whole rows; the Gram and
// update kernels stream blocks with fully coalesced accesses.
//
// Precision: T = double (FP64 mode) or float (mixed mode: FP32 factors, FP32
// accumulation inside a CTA, FP64 reduction across CTAs and FP64 H).
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "kernels.h"

namespace sylv {

int64_t& launch_counter() {
  static thread_local int64_t c = 0;
  return c;
}

namespace {

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
}

template <typename T>
struct AccOf { using type = T; };

// Vector load/store of one row of an s-wide block.
template <typename T, int S>
__device__ __forceinline__ void ld_row(const T* p, T (&v)[S]) {
  if constexpr ((S * sizeof(T)) % 16 == 0) {
#pragma unroll
    for (int i = 0; i < (int)(S * sizeof(T) / 16); ++i) {
      uint4 q = *(reinterpret_cast<const uint4*>(p) + i);
      memcpy(&v[i * 16 / sizeof(T)], &q, 16);
    }
  } else {
#pragma unroll
    for (int u = 0; u < S; ++u) v[u] = p[u];
  }
}

template <typename T, int S>
__device__ __forceinline__ void ld_row_ro(const T* __restrict__ p, T (&v)[S]) {
  if constexpr ((S * sizeof(T)) % 16 == 0) {
#pragma unroll
    for (int i = 0; i < (int)(S * sizeof(T) / 16); ++i) {
      uint4 q = __ldg(reinterpret_cast<const uint4*>(p) + i);
      memcpy(&v[i * 16 / sizeof(T)], &q, 16);
    }
  } else {
#pragma unroll
    for (int u = 0; u < S; ++u) v[u] = __ldg(p + u);
  }
}

template <typename T, int S>
__device__ __forceinline__ void st_row(T* p, const T (&v)[S]) {
  if constexpr ((S * sizeof(T)) % 16 == 0) {
#pragma unroll
    for (int i = 0; i < (int)(S * sizeof(T) / 16); ++i) {
      uint4 q;
      memcpy(&q, &v[i * 16 / sizeof(T)], 16);
      *(reinterpret_cast<uint4*>(p) + i) = q;
    }
  } else {
#pragma unroll
    for (int u = 0; u < S; ++u) p[u] = v[u];
  }
}

// Block-wide reduction of an S x S register tile into out[0..S*S) (NT threads).
template <typename A, int S>
__device__ __forceinline__ void block_reduce_tile(A (&acc)[S][S], double* out, double* sh /* (NT/32) * S*S */) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int u = 0; u < S; ++u)
#pragma unroll
    for (int t = 0; t < S; ++t) {
      A v = acc[u][t];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (l == 0) sh[w * S * S + u * S + t] = (double)v;
    }
  __syncthreads();
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += sh[i * S * S + e];
    out[e] = s;
  }
}

// Fills the lower triangle of a symmetric S x S register tile from its upper triangle (the
// self-Gram partials accumulate t >= u only: GB300's FP64 pipe is narrow).
template <typename A, int S>
__device__ __forceinline__ void mirror_upper(A (&acc)[S][S]) {
#pragma unroll
  for (int u = 1; u < S; ++u)
#pragma unroll
    for (int t = 0; t < u; ++t) acc[u][t] = acc[t][u];
}

// ---------------------------------------------------------------- SpMM
// Y = A X (- Xprev M, the three-term Lanczos term) over an s-wide block, one thread per row
// computing its s outputs.  A CTA of NT rows first stages its slice of the CSR arrays (column
// indices and values, read once and coalesced) in shared memory; each thread then walks its
// row there, gathers the s-wide rows of X as 16-byte vectors (X is small enough to stay in L2)
// and keeps s accumulators.  The s x s block M of the Lanczos term is staged in shared memory.
// A slice longer than SPMM_STAGE entries (long rows) is read from global memory instead.
// colmax (float64 only, may be null): the column maxima of |Y| as IEEE bits, combined with
// atomicMax (the digit split of the tensor-core basis).
constexpr int SPMM_STAGE = 3584;  // staged CSR entries per CTA (42 KB with float64 values: under the 48 KB static limit)

template <typename T, int S>
__global__ void __launch_bounds__(NT) spmm_kernel(const DevState* st, int64_t n, const int32_t* __restrict__ rp,
                                                  const int32_t* __restrict__ ci, const T* __restrict__ val,
                                                  const T* __restrict__ X, T* __restrict__ Y,
                                                  const T* __restrict__ Xprev, const double* __restrict__ M,
                                                  int64_t ldm, unsigned long long* __restrict__ colmax) {
  if (stopped(st)) return;
  __shared__ int32_t s_ci[SPMM_STAGE];
  __shared__ T s_val[SPMM_STAGE];
  __shared__ double s_m[S * S];
  __shared__ unsigned long long smx[S];
  const int64_t r0 = (int64_t)blockIdx.x * NT;
  const int64_t r1 = min(n, r0 + NT);
  const int64_t row = r0 + threadIdx.x;
  const int32_t p_lo = __ldg(rp + r0), p_hi = __ldg(rp + r1);
  const bool staged = p_hi - p_lo <= SPMM_STAGE;
  if (staged)
    for (int32_t p = p_lo + (int32_t)threadIdx.x; p < p_hi; p += NT) {
      s_ci[p - p_lo] = __ldg(ci + p);
      s_val[p - p_lo] = __ldg(val + p);
    }
  if (Xprev != nullptr && threadIdx.x < S * S) s_m[threadIdx.x] = M[threadIdx.x % S + (int64_t)(threadIdx.x / S) * ldm];
  if (colmax != nullptr && threadIdx.x < S) smx[threadIdx.x] = 0;
  __syncthreads();
  using A = typename AccOf<T>::type;
  A acc[S];
#pragma unroll
  for (int t = 0; t < S; ++t) acc[t] = 0;
  // Guards (the operators are square, n x n, with CSR checked on the host): a row range outside
  // the CTA's slice or a column index outside [0, n) is recorded in the status word (site 300,
  // 301) and the entry is skipped, never dereferenced.
  bool bad = false;
  if (row < n) {
    const int32_t q0 = __ldg(rp + row), q1 = __ldg(rp + row + 1);
    T x[S];
    if (staged) {
      if (q0 < p_lo || q1 > p_hi || q1 < q0) {
        bad = true;
      } else {
        for (int32_t p = q0 - p_lo; p < q1 - p_lo; ++p) {
          const int32_t c = s_ci[p];
          if (c < 0 || (int64_t)c >= n) {
            bad = true;
            continue;
          }
          ld_row_ro<T, S>(X + (int64_t)c * S, x);
          const A v = (A)s_val[p];
#pragma unroll
          for (int t = 0; t < S; ++t) acc[t] += v * (A)x[t];
        }
      }
    } else {
      for (int32_t p = q0; p < q1; ++p) {
        const int32_t c = __ldg(ci + p);
        if (c < 0 || (int64_t)c >= n) {
          bad = true;
          continue;
        }
        ld_row_ro<T, S>(X + (int64_t)c * S, x);
        const A v = (A)__ldg(val + p);
#pragma unroll
        for (int t = 0; t < S; ++t) acc[t] += v * (A)x[t];
      }
    }
    if (Xprev != nullptr) {
      ld_row_ro<T, S>(Xprev + row * S, x);
#pragma unroll
      for (int t = 0; t < S; ++t)
#pragma unroll
        for (int u = 0; u < S; ++u) acc[t] -= (A)x[u] * (A)s_m[u + t * S];
    }
    T y[S];
#pragma unroll
    for (int t = 0; t < S; ++t) y[t] = (T)acc[t];
    st_row<T, S>(Y + row * S, y);
  }
  if (bad && st != nullptr) {
    DevState* ws = const_cast<DevState*>(st);
    ws->breakdown_where = staged ? 300 : 301;
    atomicExch(&ws->status, (int)ST_BREAKDOWN);
  }
  if (colmax != nullptr) {
    if (row < n) {
#pragma unroll
      for (int t = 0; t < S; ++t) atomicMax(&smx[t], (unsigned long long)__double_as_longlong(fabs((double)acc[t])));
    }
    __syncthreads();
    if (threadIdx.x < S && smx[threadIdx.x]) atomicMax(colmax + threadIdx.x, smx[threadIdx.x]);
  }
}

// ---------------------------------------------------------------- Gram (TSGEMM)
// CTA c owns rows [c*rpc, (c+1)*rpc).  Warp tasks = (block b, row slice); a task
// streams V_b over its rows (lanes = consecutive rows, coalesced), accumulates the
// S x S tile V_b^T Y in registers, reduces it across the warp and writes it.
// When there are fewer blocks than warps, rows are split into slices and the
// slice tiles are summed through shared memory in a fixed order.
template <typename T, int S>
__global__ void __launch_bounds__(NT) gram_kernel(const DevState* st, int64_t n, int64_t rpc, const T* __restrict__ V,
                                                  int64_t bstride, int nb, const T* __restrict__ Y,
                                                  T* __restrict__ partial) {
  if (stopped(st)) return;
  // partials stay in the factor precision (float in the mixed mode): converting them
  // to double here would occupy GB300's narrow FP64 pipe; the reduce kernel does it
  __shared__ T sh[(NT / 32) * S * S];
  using A = typename AccOf<T>::type;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = NT / 32;
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int64_t r1 = min(n, r0 + rpc);
  const int slices = nb >= nw ? 1 : nw / nb;
  const int ntasks = nb * slices;
  T* out = partial + (int64_t)blockIdx.x * nb * S * S;
  for (int task = w; task < ntasks; task += nw) {
    const int b = task / slices, sl = task - b * slices;
    const T* Vb = V + (int64_t)b * bstride;
    A acc[S][S];
#pragma unroll
    for (int u = 0; u < S; ++u)
#pragma unroll
      for (int t = 0; t < S; ++t) acc[u][t] = 0;
    // UNR independent rows per lane in flight (more bytes in flight per warp for the
    // HBM-bound FP32 case; bounded so the S x S accumulators stay in registers)
    constexpr int RB = S * (int)sizeof(T);
    constexpr int UNR = RB <= 16 ? 4 : (RB <= 32 ? 2 : 1);
    const int64_t step = 32 * (int64_t)slices;
    int64_t row = r0 + (int64_t)sl * 32 + l;
    for (; row + (UNR - 1) * step < r1; row += UNR * step) {
      T v[UNR][S], y[UNR][S];
#pragma unroll
      for (int q = 0; q < UNR; ++q) {
        ld_row_ro<T, S>(Vb + (row + q * step) * S, v[q]);
        ld_row<T, S>(Y + (row + q * step) * S, y[q]);
      }
#pragma unroll
      for (int q = 0; q < UNR; ++q)
#pragma unroll
        for (int u = 0; u < S; ++u)
#pragma unroll
          for (int t = 0; t < S; ++t) acc[u][t] += (A)v[q][u] * (A)y[q][t];
    }
    for (; row < r1; row += step) {
      T v[S], y[S];
      ld_row_ro<T, S>(Vb + row * S, v);
      ld_row<T, S>(Y + row * S, y);
#pragma unroll
      for (int u = 0; u < S; ++u)
#pragma unroll
        for (int t = 0; t < S; ++t) acc[u][t] += (A)v[u] * (A)y[t];
    }
#pragma unroll
    for (int u = 0; u < S; ++u)
#pragma unroll
      for (int t = 0; t < S; ++t) {
        A v = acc[u][t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int e = u * S + t;
        if (slices == 1) {
          if (l == (e & 31)) out[b * S * S + e] = (T)v;
        } else {
          if (l == (e & 31)) sh[task * S * S + e] = (T)v;
        }
      }
  }
  if (slices > 1) {
    __syncthreads();
    for (int e = threadIdx.x; e < nb * S * S; e += NT) {
      const int b = e / (S * S), r = e - b * S * S;
      T s = 0;
      for (int sl = 0; sl < slices; ++sl) s += sh[(b * slices + sl) * S * S + r];
      out[e] = s;
    }
  }
}

// Fixed-order sum of the per-CTA partials.  A CTA covers 8 outputs; 32 groups of threads
// split each output's partials (group g takes CTAs g, g+32, ...), so every thread has only
// ncta/32 loads in its chain (the sum is latency-bound, not bandwidth-bound), and the 32
// group sums are added in a fixed order.
constexpr int RED_E = 8, RED_G = 32;

template <typename P>
__global__ void __launch_bounds__(RED_E * RED_G) reduce_H_kernel(const DevState* st, const P* __restrict__ partial,
                                                                 int ncta, int nb, int s, double* __restrict__ H,
                                                                 int64_t ldh, int64_t row0, int64_t col0,
                                                                 double* __restrict__ Hc, int add) {
  if (stopped(st)) return;
  __shared__ double part[RED_G][RED_E];
  const int E = nb * s * s;
  const int el = threadIdx.x % RED_E, g = threadIdx.x / RED_E;
  const int e = blockIdx.x * RED_E + el;
  double v0 = 0.0, v1 = 0.0;
  if (e < E) {
    int c = g;
    for (; c + RED_G < ncta; c += 2 * RED_G) {
      v0 += (double)partial[(int64_t)c * E + e];
      v1 += (double)partial[(int64_t)(c + RED_G) * E + e];
    }
    if (c < ncta) v0 += (double)partial[(int64_t)c * E + e];
  }
  part[g][el] = v0 + v1;
  __syncthreads();
  if (g != 0 || e >= E) return;
  double vs = 0.0;
  for (int q = 0; q < RED_G; ++q) vs += part[q][el];
  Hc[e] = vs;
  const int b = e / (s * s), r = e - b * s * s, u = r / s, t = r - u * s;
  double* h = H + (row0 + (int64_t)b * s + u) + (col0 + t) * ldh;
  *h = add ? (*h + vs) : vs;
}

// ---------------------------------------------------------------- block update
// One thread per row (grid-stride): y -= sum_b V_b[row] Hc_b, with Hc staged in
// shared memory in chunks; optionally accumulates the partial Y^T Y of the result.
template <typename T, int S>
constexpr int upd_chunk() {
  return (int)std::max<size_t>(1, (32 * 1024) / (S * S * sizeof(T)));
}

template <typename T, int S, bool SELF>
__global__ void __launch_bounds__(NT) update_kernel(const DevState* st, int64_t n, const T* __restrict__ V,
                                                    int64_t bstride, int nb, const double* __restrict__ Hc,
                                                    T* __restrict__ Y, double* __restrict__ partial) {
  if (stopped(st)) return;
  constexpr int CH = upd_chunk<T, S>();
  __shared__ __align__(16) T hs[CH * S * S];
  __shared__ double sh[(NT / 32) * S * S];
  using A = typename AccOf<T>::type;
  A acc[S][S];
  if constexpr (SELF) {
#pragma unroll
    for (int u = 0; u < S; ++u)
#pragma unroll
      for (int t = 0; t < S; ++t) acc[u][t] = 0;
  }
  for (int64_t base = (int64_t)blockIdx.x * NT; base < n; base += (int64_t)gridDim.x * NT) {
    const int64_t row = base + threadIdx.x;
    T y[S];
    if (row < n) ld_row<T, S>(Y + row * S, y);
    for (int b0 = 0; b0 < nb; b0 += CH) {
      const int cb = min(CH, nb - b0);
      __syncthreads();
      for (int e = threadIdx.x; e < cb * S * S; e += NT) hs[e] = (T)Hc[(int64_t)b0 * S * S + e];
      __syncthreads();
      if (row < n) {
#pragma unroll 4
        for (int b = 0; b < cb; ++b) {
          T v[S];
          ld_row_ro<T, S>(V + (int64_t)(b0 + b) * bstride + row * S, v);
#pragma unroll
          for (int u = 0; u < S; ++u)
#pragma unroll
            for (int t = 0; t < S; ++t) y[t] -= v[u] * hs[(b * S + u) * S + t];
        }
      }
    }
    if (row < n) {
      st_row<T, S>(Y + row * S, y);
      if constexpr (SELF) {
#pragma unroll
        for (int u = 0; u < S; ++u)
#pragma unroll
          for (int t = u; t < S; ++t) acc[u][t] += (A)y[u] * (A)y[t];  // upper triangle
      }
    }
  }
  if constexpr (SELF) {
    mirror_upper<A, S>(acc);
    block_reduce_tile<A, S>(acc, partial + (int64_t)blockIdx.x * S * S, sh);
  }
}

template <typename T, int S>
__global__ void __launch_bounds__(NT) selfgram_kernel(const DevState* st, int64_t n, const T* __restrict__ Y,
                                                      double* __restrict__ partial) {
  if (stopped(st)) return;
  __shared__ double sh[(NT / 32) * S * S];
  using A = typename AccOf<T>::type;
  A acc[S][S];
#pragma unroll
  for (int u = 0; u < S; ++u)
#pragma unroll
    for (int t = 0; t < S; ++t) acc[u][t] = 0;
  for (int64_t row = (int64_t)blockIdx.x * NT + threadIdx.x; row < n; row += (int64_t)gridDim.x * NT) {
    T y[S];
    ld_row<T, S>(Y + row * S, y);
#pragma unroll
    for (int u = 0; u < S; ++u)
#pragma unroll
      for (int t = u; t < S; ++t) acc[u][t] += (A)y[u] * (A)y[t];  // upper triangle
  }
  mirror_upper<A, S>(acc);
  block_reduce_tile<A, S>(acc, partial + (int64_t)blockIdx.x * S * S, sh);
}


// ---------------------------------------------------------------- CholQR pass
// Single CTA: G = sum of the partial Gram tiles; nu^2 = ||H_{1:j,j}||^2 + tr(G);
// exhaustion if tr(G) <= delta^2 nu^2 (the block becomes zero); Cholesky G = R^T R
// (upper R, positive diagonal); a pivot <= (delta nu)^2 on pass 1 is a partial loss
// of rank (breakdown).  Writes R^{-1} for the scale kernel and, on pass 2,
// H_{j+1,j} = R2 R1.
// CTA-level: every CTA that calls it computes the same factors (same inputs, same order of
// operations); `writer` CTAs also store them.  Leaves R^{-1} in Ri_out (shared memory) and
// returns 1 when the block is to be scaled (0 after a breakdown or a non-finite value).
__device__ int chol_block(DevState* st, const double* __restrict__ partial, int ncta, const CholArgs& a, bool writer,
                          double* Ri_out) {
  __shared__ double G[64], R[64], Ri[64], sh[32];
  __shared__ double gsum[NT];
  const int s = a.s, E = s * s;
  {
    // thread -> (entry e, group g); each group sums a strided subset of the CTA
    // partials, then the groups are added in a fixed order (deterministic)
    const int groups = NT / E;
    const int e = threadIdx.x % E, g = threadIdx.x / E;
    double v = 0.0;
    if (g < groups) {
      double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
      int c = g;
      for (; c + 3 * groups < ncta; c += 4 * groups) {
        v0 += partial[(int64_t)c * E + e];
        v1 += partial[(int64_t)(c + groups) * E + e];
        v2 += partial[(int64_t)(c + 2 * groups) * E + e];
        v3 += partial[(int64_t)(c + 3 * groups) * E + e];
      }
      for (; c < ncta; c += groups) v0 += partial[(int64_t)c * E + e];
      v = (v0 + v1) + (v2 + v3);
    }
    gsum[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < E) {
      double t = 0.0;
      for (int q = 0; q < groups; ++q) t += gsum[q * E + threadIdx.x];
      G[threadIdx.x] = t;
    }
    __syncthreads();
  }
  double hsq = 0.0;
  if (a.pass == 1 && a.Hcol != nullptr) {  // ||H_{1:j,j}||^2, four independent chains per thread
    double h0 = 0.0, h1 = 0.0, h2 = 0.0, h3 = 0.0;
    for (int t = 0; t < s; ++t) {
      const double* col = a.Hcol + (int64_t)t * a.ldh;
      int64_t i = threadIdx.x;
      for (; i + 3 * NT < a.hrows; i += 4 * NT) {
        const double x0 = col[i], x1 = col[i + NT], x2 = col[i + 2 * NT], x3 = col[i + 3 * NT];
        h0 += x0 * x0;
        h1 += x1 * x1;
        h2 += x2 * x2;
        h3 += x3 * x3;
      }
      for (; i < a.hrows; i += NT) h0 += col[i] * col[i];
    }
    hsq = (h0 + h1) + (h2 + h3);
  }
  hsq = block_sum(hsq, sh);
  // The s x s factorisation runs on one warp with the lanes in parallel: on this GPU every
  // float64 instruction of a single thread holds the FP64 pipe of its quarter-SM for tens of
  // cycles, so a one-thread Cholesky + inverse + product took ~20 us.  Shared memory holds
  // the Schur complement S, R, R^-1, 1/R_jj, R1 (pass 2) and the product R2 R1.
  __shared__ double R1s[64], Pm[64], S[64], dinv[8];
  __shared__ int out_sh;  // 0: write nothing, 1: write the factors (zero ones if exhausted)
  if (threadIdx.x < 64) {
    R[threadIdx.x] = 0.0;
    Ri[threadIdx.x] = 0.0;
    Pm[threadIdx.x] = 0.0;
    if (threadIdx.x < 8) dinv[threadIdx.x] = 0.0;
    S[threadIdx.x] = threadIdx.x < E ? G[threadIdx.x] : 0.0;
    R1s[threadIdx.x] = (a.pass == 2 && threadIdx.x < E) ? a.R1[threadIdx.x] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    bool finite = true;
    for (int e = lane; e < E; e += 32) finite = finite && isfinite(G[e]);
    finite = __all_sync(0xffffffffu, finite);
    double tr = 0.0;  // G[u*s+t] = sum_rows y_u y_t (symmetric)
    for (int u = 0; u < s; ++u) tr += G[u * s + u];
    const double nu2 = hsq + tr;
    int exh = (a.pass == 2) ? st->exhausted[a.side] : 0;
    int bad = 0;
    if (!finite || !isfinite(hsq)) {
      bad = 1;
      if (lane == 0) {
        st->status = ST_NONFINITE;
        st->breakdown_where = 100 + a.side;
      }
    } else if (a.pass == 1 && !a.setup && tr <= a.delta * a.delta * nu2) {
      exh = 1;
      if (lane == 0) st->exhausted[a.side] = 1;
    }
    if (!bad && !exh) {
      // right-looking Cholesky G = R^T R (upper R, positive diagonal); the updates of each
      // entry subtract the same terms in the same order as the left-looking form.  A pivot
      // <= thr is a column (numerically) dependent on the earlier ones: it is deflated -- its
      // R row, R^-1 row and column stay zero, so its basis column becomes zero and stays zero
      // in every later block -- except in the QR of C1, C2, where it is a breakdown.
      const double thr = (a.pass == 1) ? a.delta * a.delta * nu2 : 0.0;
      for (int j = 0; j < s; ++j) {
        const double d = S[j * s + j];
        if (!(d > thr)) {  // the same value in every lane: a uniform branch
          if (a.setup) {
            bad = 1;
            if (lane == 0) {
              st->status = ST_BREAKDOWN;
              st->breakdown_where = 10 + a.side;
            }
            break;
          }
          continue;
        }
        const double rjj = sqrt(d), rinv = 1.0 / rjj;
        if (lane == j) {
          R[j + j * s] = rjj;
          dinv[j] = rinv;
        } else if (lane > j && lane < s) {
          R[j + lane * s] = S[j * s + lane] * rinv;
        }
        __syncwarp();
        const int m = s - j - 1;
        for (int p = lane; p < m * m; p += 32) {
          const int i = j + 1 + p / m, l = j + 1 + p % m;
          S[i * s + l] -= R[j + i * s] * R[j + l * s];
        }
        __syncwarp();
      }
      if (!bad) {
        // R^-1 column by column; the rows of a column in parallel
        for (int j = 0; j < s; ++j) {
          if (lane == j) {
            Ri[j + j * s] = dinv[j];
          } else if (lane < j) {
            double acc = 0.0;
            for (int k = lane; k < j; ++k) acc += Ri[lane + k * s] * R[k + j * s];
            Ri[lane + j * s] = -acc * dinv[j];
          }
          __syncwarp();
        }
      }
    }
    if (!bad && a.pass == 2) {  // R2 R1 (both upper triangular)
      for (int e = lane; e < E; e += 32) {
        const int i = e % s, j = e / s;
        double acc = 0.0;
        for (int k = 0; k < s; ++k) acc += R[i + k * s] * R1s[k + j * s];
        Pm[e] = exh ? 0.0 : acc;
      }
    }
    if (lane == 0) out_sh = bad ? 0 : 1;
  }
  __syncthreads();
  const int e = threadIdx.x;
  const int out = out_sh;
  if (e < 64) Ri_out[e] = Ri[e];
  if (writer && out != 0 && e < E) {
    a.Rinv[e] = Ri[e];
    if (a.factor_is_float)
      ((float*)a.RinvT)[e] = (float)Ri[e];
    else
      ((double*)a.RinvT)[e] = Ri[e];
    if (a.pass == 1) {
      a.R1[e] = R[e];
    } else {
      const int i = e % s, j = e / s;
      if (a.Hsub) a.Hsub[i + j * a.ldh] = Pm[e];
      if (a.Hsup) a.Hsup[j + i * a.ldh] = Pm[e];
      if (a.Rout) a.Rout[e] = Pm[e];
    }
  }
  __syncthreads();
  return out;
}


// One CholQR pass in one launch: every CTA forms the s x s Gram from the partials of the
// previous kernel and factors it (chol_block: the same factors in every CTA; CTA 0 stores
// them), then scales its rows, Y <- Y R^{-1}, with the optional partial Y^T Y of the result
// (SELF, into partial_out, which must not be partial_in) and column maxima (colmax).
template <typename T, int S, bool SELF>
__global__ void __launch_bounds__(NT) cholscale_kernel(DevState* st, const double* __restrict__ partial_in,
                                                       int ncta_in, CholArgs a, int64_t n, T* __restrict__ Y,
                                                       double* __restrict__ partial_out,
                                                       unsigned long long* __restrict__ colmax) {
  if (stopped(st)) return;
  __shared__ double Rid[64];
  __shared__ T rs[S * S];
  __shared__ double sh[(NT / 32) * S * S];
  __shared__ unsigned long long smx[S];
  if (!chol_block(st, partial_in, ncta_in, a, blockIdx.x == 0, Rid)) return;  // uniform in the CTA
  if (threadIdx.x < S * S) rs[threadIdx.x] = (T)Rid[(threadIdx.x % S) + (threadIdx.x / S) * S];
  if (threadIdx.x < S) smx[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long zmax[S];
#pragma unroll
  for (int t = 0; t < S; ++t) zmax[t] = 0;
  using A = typename AccOf<T>::type;
  A acc[S][S];
  if constexpr (SELF) {
#pragma unroll
    for (int u = 0; u < S; ++u)
#pragma unroll
      for (int t = 0; t < S; ++t) acc[u][t] = 0;
  }
  for (int64_t row = (int64_t)blockIdx.x * NT + threadIdx.x; row < n; row += (int64_t)gridDim.x * NT) {
    T y[S], z[S];
    ld_row<T, S>(Y + row * S, y);
#pragma unroll
    for (int t = 0; t < S; ++t) {
      T v = 0;
#pragma unroll
      for (int u = 0; u <= t; ++u) v += y[u] * rs[u + t * S];
      z[t] = v;
    }
    st_row<T, S>(Y + row * S, z);
    if constexpr (SELF) {
#pragma unroll
      for (int u = 0; u < S; ++u)
#pragma unroll
        for (int t = u; t < S; ++t) acc[u][t] += (A)z[u] * (A)z[t];  // upper triangle
    }
    if (colmax != nullptr) {
#pragma unroll
      for (int t = 0; t < S; ++t)
        zmax[t] = max(zmax[t], (unsigned long long)__double_as_longlong(fabs((double)z[t])));
    }
  }
  if constexpr (SELF) {
    mirror_upper<A, S>(acc);
    block_reduce_tile<A, S>(acc, partial_out + (int64_t)blockIdx.x * S * S, sh);
  }
  if (colmax != nullptr) {
#pragma unroll
    for (int t = 0; t < S; ++t) {
      unsigned long long v = zmax[t];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
      if ((threadIdx.x & 31) == 0 && v) atomicMax(&smx[t], v);
    }
    __syncthreads();
    if (threadIdx.x < S && smx[threadIdx.x]) atomicMax(colmax + threadIdx.x, smx[threadIdx.x]);
  }
}

// ---------------------------------------------------------------- layout helpers
template <typename T, int S>
__global__ void pack_kernel(int64_t n, const double* __restrict__ Ccol, T* __restrict__ V) {
  const int64_t gid = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (gid >= n * S) return;
  const int64_t row = gid / S;
  const int t = (int)(gid - row * S);
  V[gid] = (T)Ccol[row + t * n];
}

template <typename T>
__global__ void unpack_kernel(int64_t n, int s, int64_t total, const T* __restrict__ V, int64_t bstride,
                              double* __restrict__ Vcol) {
  const int64_t gid = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (gid >= total) return;
  const int64_t col = gid / n, row = gid - col * n;
  const int64_t b = col / s, t = col - b * s;
  Vcol[gid] = (double)V[b * bstride + row * s + t];
}

template <typename T>
__global__ void convert_kernel(int64_t count, const double* __restrict__ src, T* __restrict__ dst) {
  const int64_t gid = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (gid < count) dst[gid] = (T)src[gid];
}

int grid_for(int64_t work, int64_t per, int cap) {
  int64_t g = (work + per - 1) / per;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

#define SYLV_S_CASES(MACRO) \
  MACRO(1) MACRO(2) MACRO(3) MACRO(4) MACRO(5) MACRO(6) MACRO(7) MACRO(8)

template <typename T>
void launch_spmm(cudaStream_t strm, const DevState* st, int64_t n, int s, const int32_t* rp, const int32_t* ci,
                 const T* val, const T* X, T* Y, const T* Xprev, const double* M, int64_t ldm,
                 unsigned long long* colmax) {
  const int grid = (int)((n + NT - 1) / NT);  // one thread per row
  if (grid == 0) return;
#define CASE(SV) \
  case SV: spmm_kernel<T, SV><<<counted(grid), NT, 0, strm>>>(st, n, rp, ci, val, X, Y, Xprev, M, ldm, colmax); break;
  switch (s) { SYLV_S_CASES(CASE) }
#undef CASE
}

template <typename T>
int launch_gram(cudaStream_t strm, const DevState* st, int64_t n, int s, const T* V, int64_t bstride, int nb,
                const T* Y, double* partial) {
  // FP64 is bound by the FP64 pipe: one CTA per SM keeps the per-task warp
  // reductions (s*s shuffle+add steps) small next to the row loop.  FP32 is bound
  // by HBM latency: four CTAs per SM for more loads in flight.  The partials are
  // written in the factor precision (T), read by launch_reduce_H<T>.
  const int grid = grid_for(n, 64, (sizeof(T) == 8 ? 1 : 4) * num_sms());
  const int64_t rpc = (n + grid - 1) / grid;
  T* tpart = reinterpret_cast<T*>(partial);
#define CASE(SV) \
  case SV: gram_kernel<T, SV><<<counted(grid), NT, 0, strm>>>(st, n, rpc, V, bstride, nb, Y, tpart); break;
  switch (s) { SYLV_S_CASES(CASE) }
#undef CASE
  return grid;
}

void launch_reduce_H(cudaStream_t strm, const DevState* st, const double* partial, int ncta, int nb, int s, double* H,
                     int64_t ldh, int64_t row0, int64_t col0, double* Hc, bool add, bool float_partials) {
  const int E = nb * s * s;
  const int grid = (E + RED_E - 1) / RED_E;
  if (float_partials)
    reduce_H_kernel<float><<<counted(grid), RED_E * RED_G, 0, strm>>>(st, reinterpret_cast<const float*>(partial), ncta, nb, s,
                                                             H, ldh, row0, col0, Hc, add ? 1 : 0);
  else
    reduce_H_kernel<double><<<counted(grid), RED_E * RED_G, 0, strm>>>(st, partial, ncta, nb, s, H, ldh, row0, col0, Hc,
                                                              add ? 1 : 0);
}

template <typename T>
int launch_update(cudaStream_t strm, const DevState* st, int64_t n, int s, const T* V, int64_t bstride, int nb,
                  const double* Hc, T* Y, double* self_partial) {
  const int grid = grid_for(n, NT, 4 * num_sms());
#define CASE(SV)                                                                                         \
  case SV:                                                                                               \
    if (self_partial)                                                                                    \
      update_kernel<T, SV, true><<<counted(grid), NT, 0, strm>>>(st, n, V, bstride, nb, Hc, Y, self_partial);     \
    else                                                                                                 \
      update_kernel<T, SV, false><<<counted(grid), NT, 0, strm>>>(st, n, V, bstride, nb, Hc, Y, nullptr);         \
    break;
  switch (s) { SYLV_S_CASES(CASE) }
#undef CASE
  return grid;
}

template <typename T>
int launch_selfgram(cudaStream_t strm, const DevState* st, int64_t n, int s, const T* Y, double* self_partial) {
  const int grid = grid_for(n, NT, 4 * num_sms());
#define CASE(SV) \
  case SV: selfgram_kernel<T, SV><<<counted(grid), NT, 0, strm>>>(st, n, Y, self_partial); break;
  switch (s) { SYLV_S_CASES(CASE) }
#undef CASE
  return grid;
}



template <typename T>
int launch_cholscale(cudaStream_t strm, DevState* st, const double* partial_in, int ncta_in, const CholArgs& a,
                     int64_t n, T* Y, double* partial_out, unsigned long long* colmax) {
  // two CTAs per SM: every CTA also reduces the ncta_in partials and factors the s x s Gram
  const int grid = grid_for(n, NT, 2 * num_sms());
#define CASE(SV)                                                                                                    \
  case SV:                                                                                                          \
    if (partial_out)                                                                                                \
      cholscale_kernel<T, SV, true><<<counted(grid), NT, 0, strm>>>(st, partial_in, ncta_in, a, n, Y, partial_out,  \
                                                                    colmax);                                        \
    else                                                                                                            \
      cholscale_kernel<T, SV, false><<<counted(grid), NT, 0, strm>>>(st, partial_in, ncta_in, a, n, Y, nullptr,     \
                                                                     colmax);                                       \
    break;
  switch (a.s) { SYLV_S_CASES(CASE) }
#undef CASE
  return grid;
}

template <typename T>
void launch_pack(cudaStream_t strm, int64_t n, int s, const double* Ccol, T* Vblk) {
  const int grid = (int)((n * s + NT - 1) / NT);
  if (grid == 0) return;
#define CASE(SV) \
  case SV: pack_kernel<T, SV><<<counted(grid), NT, 0, strm>>>(n, Ccol, Vblk); break;
  switch (s) { SYLV_S_CASES(CASE) }
#undef CASE
}

template <typename T>
void launch_unpack(cudaStream_t strm, int64_t n, int s, int nb, const T* Vblk, int64_t bstride, double* Vcol) {
  const int64_t total = n * s * (int64_t)nb;
  if (total == 0) return;
  unpack_kernel<T><<<counted((unsigned)((total + NT - 1) / NT)), NT, 0, strm>>>(n, s, total, Vblk, bstride, Vcol);
}

template <typename T>
void launch_convert(cudaStream_t strm, int64_t count, const double* src, T* dst) {
  if (count == 0) return;
  convert_kernel<T><<<counted((unsigned)((count + NT - 1) / NT)), NT, 0, strm>>>(count, src, dst);
}

#define SYLV_INST(T)                                                                                              \
  template void launch_spmm<T>(cudaStream_t, const DevState*, int64_t, int, const int32_t*, const int32_t*,      \
                               const T*, const T*, T*, const T*, const double*, int64_t, unsigned long long*);   \
  template int launch_gram<T>(cudaStream_t, const DevState*, int64_t, int, const T*, int64_t, int, const T*,     \
                              double*);                                                                          \
  template int launch_update<T>(cudaStream_t, const DevState*, int64_t, int, const T*, int64_t, int,             \
                                const double*, T*, double*);                                                     \
  template int launch_selfgram<T>(cudaStream_t, const DevState*, int64_t, int, const T*, double*);               \
  template int launch_cholscale<T>(cudaStream_t, DevState*, const double*, int, const CholArgs&, int64_t, T*,    \
                                   double*, unsigned long long*);                                                \
  template void launch_pack<T>(cudaStream_t, int64_t, int, const double*, T*);                                  \
  template void launch_unpack<T>(cudaStream_t, int64_t, int, int, const T*, int64_t, double*);                  \
  template void launch_convert<T>(cudaStream_t, int64_t, const double*, T*);

SYLV_INST(double)
SYLV_INST(float)

}  // namespace sylv
