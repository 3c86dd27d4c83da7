// Final low-rank compression of the factored iterate X = V X^ W^T (float64).
//
// With orthonormal V, W (the float64 block Arnoldi bases; deflated zero columns allowed --
// their rows and columns of X^ are zero) the singular values of X are those of X^, so
// X^ = U S Z^T gives X = (V U) S (W Z)^T, and keeping the q largest singular values is the
// best rank-q approximation (Eckart-Young).  The SVD of the r x r core is a one-sided
// (Hestenes) Jacobi iteration: rounds of r/2 disjoint column pairs (a round-robin schedule,
// every pair once per sweep), one CTA per pair, each rotating the two columns of G (initially
// X^) and of Z (initially I) so that they become orthogonal (Rutishauser's formulas for the
// rotation); sweeps repeat until a sweep rotates nothing.  Then s_i = ||g_i||, U = G S^-1.
// Columns with ||g||^2 <= tau, tau = (r eps ||X^||_F)^2, are at the rounding floor: their
// directions are noise that never settles, so pairs with such a column are not rotated (their
// singular values are below that floor and any tolerance above it truncates them).
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace sylv {

namespace {

// One Jacobi round: CTA p takes the pair (pairs[2p], pairs[2p+1]) (an index -1: no partner).
__global__ void __launch_bounds__(NT) jacobi_round_kernel(int r, double* __restrict__ G, double* __restrict__ Z,
                                                          int64_t ld, const int* __restrict__ pairs, double eps,
                                                          double tau, int* __restrict__ rotated) {
  __shared__ double sh[32];
  __shared__ double rot[2];
  __shared__ int do_sh;
  const int i = pairs[2 * blockIdx.x], j = pairs[2 * blockIdx.x + 1];
  if (i < 0 || j < 0) return;
  double* gi = G + (int64_t)i * ld;
  double* gj = G + (int64_t)j * ld;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int k = threadIdx.x; k < r; k += NT) {
    const double x = gi[k], y = gj[k];
    a += x * x;
    b += y * y;
    c += x * y;
  }
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  c = block_sum(c, sh);
  if (threadIdx.x == 0) {
    do_sh = 0;
    if (a > tau && b > tau && fabs(c) > eps * sqrt(a) * sqrt(b)) {
      const double zeta = (b - a) / (2.0 * c);
      const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      const double cs = 1.0 / sqrt(1.0 + t * t);
      rot[0] = cs;
      rot[1] = cs * t;
      do_sh = 1;
      atomicAdd(rotated, 1);
    }
  }
  __syncthreads();
  if (!do_sh) return;
  const double cs = rot[0], sn = rot[1];
  double* zi = Z + (int64_t)i * ld;
  double* zj = Z + (int64_t)j * ld;
  for (int k = threadIdx.x; k < r; k += NT) {
    const double x = gi[k], y = gj[k];
    gi[k] = cs * x - sn * y;
    gj[k] = sn * x + cs * y;
    const double u = zi[k], v = zj[k];
    zi[k] = cs * u - sn * v;
    zj[k] = sn * u + cs * v;
  }
}

// s[i] = ||g_i|| (one CTA per column)
__global__ void __launch_bounds__(NT) column_norms_kernel(int r, const double* __restrict__ G, int64_t ld,
                                                          double* __restrict__ s) {
  __shared__ double sh[32];
  const double* g = G + (int64_t)blockIdx.x * ld;
  double a = 0.0;
  for (int k = threadIdx.x; k < r; k += NT) a += g[k] * g[k];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) s[blockIdx.x] = sqrt(a);
}

// Out (rows x q, column-major, ld rows) = Vblk (rows x r, nb blocks of width su, block-row-major)
// times M(:, cols[0..q)) scaled column-wise by scale[0..q) (M: r x r column-major, ld ldm).
constexpr int AB_COLS = 8, AB_K = 64;
__global__ void __launch_bounds__(NT) apply_blocks_kernel(int64_t rows, int su, int r, const double* __restrict__ V,
                                                          int64_t bstride, const double* __restrict__ M, int64_t ldm,
                                                          const int* __restrict__ cols, const double* __restrict__ scale,
                                                          int q, double* __restrict__ Out) {
  __shared__ double ms[AB_K][AB_COLS];
  const int64_t row = (int64_t)blockIdx.x * NT + threadIdx.x;
  const int c0 = blockIdx.y * AB_COLS;
  double acc[AB_COLS];
#pragma unroll
  for (int t = 0; t < AB_COLS; ++t) acc[t] = 0.0;
  int b = 0, u = 0;  // (block, column) of k
  for (int k0 = 0; k0 < r; k0 += AB_K) {
    const int kc = min(AB_K, r - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < AB_K * AB_COLS; e += NT) {
      const int kk = e / AB_COLS, t = e % AB_COLS;
      double v = 0.0;
      if (kk < kc && c0 + t < q) v = M[(k0 + kk) + (int64_t)cols[c0 + t] * ldm] * scale[c0 + t];
      ms[kk][t] = v;
    }
    __syncthreads();
    if (row < rows) {
      for (int kk = 0; kk < kc; ++kk) {
        const double v = V[(int64_t)b * bstride + row * su + u];
#pragma unroll
        for (int t = 0; t < AB_COLS; ++t) acc[t] += v * ms[kk][t];
        if (++u == su) {
          u = 0;
          ++b;
        }
      }
    }
  }
  if (row < rows) {
#pragma unroll
    for (int t = 0; t < AB_COLS; ++t)
      if (c0 + t < q) Out[row + (int64_t)(c0 + t) * rows] = acc[t];
  }
}

}  // namespace

// Round-robin schedule (circle method) of all pairs of r columns: r2 - 1 rounds of r2 / 2 pairs
// (r2 = r rounded up to even; the extra index is -1).  pairs has (r2 - 1) * r2 entries.
void jacobi_schedule(int r, std::vector<int>& pairs) {
  const int r2 = r + (r & 1);
  std::vector<int> ring(r2);
  for (int i = 0; i < r2; ++i) ring[i] = i < r ? i : -1;
  pairs.clear();
  for (int round = 0; round < r2 - 1; ++round) {
    for (int p = 0; p < r2 / 2; ++p) {
      const int x = ring[p], y = ring[r2 - 1 - p];
      pairs.push_back(std::min(x, y) < 0 ? -1 : std::min(x, y));
      pairs.push_back(std::min(x, y) < 0 ? -1 : std::max(x, y));
    }
    // keep ring[0], rotate the rest by one
    const int last = ring[r2 - 1];
    for (int i = r2 - 1; i > 1; --i) ring[i] = ring[i - 1];
    ring[1] = last;
  }
}

int launch_jacobi_round(cudaStream_t strm, int r, double* G, double* Z, int64_t ld, const int* pairs_round,
                        double eps, double tau, int* rotated) {
  const int np = (r + (r & 1)) / 2;
  if (np == 0) return 0;
  jacobi_round_kernel<<<counted(np), NT, 0, strm>>>(r, G, Z, ld, pairs_round, eps, tau, rotated);
  return 1;
}

void launch_column_norms(cudaStream_t strm, int r, const double* G, int64_t ld, double* s) {
  if (r == 0) return;
  column_norms_kernel<<<counted(r), NT, 0, strm>>>(r, G, ld, s);
}

void launch_apply_blocks(cudaStream_t strm, int64_t rows, int su, int r, const double* V, int64_t bstride,
                         const double* M, int64_t ldm, const int* cols, const double* scale, int q, double* Out) {
  if (rows == 0 || q == 0) return;
  const dim3 g((unsigned)((rows + NT - 1) / NT), (unsigned)((q + AB_COLS - 1) / AB_COLS));
  apply_blocks_kernel<<<counted(g), NT, 0, strm>>>(rows, su, r, V, bstride, M, ldm, cols, scale, q, Out);
}

}  // namespace sylv
