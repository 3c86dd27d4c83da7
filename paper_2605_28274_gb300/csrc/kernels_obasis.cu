// Float64-accurate block Gram products and block updates of the Arnoldi bases on the tcgen05
// tensor cores.
//
// In the float64 solve the basis kernels of eq. 3.4 -- H_{1:j,j} = V^T Y and Y -= V H_{1:j,j},
// each twice per step in block classical Gram-Schmidt -- do 2 s flops per basis element they
// read.  GB300 executes float64 FMAs at 1/64 of its FP32 rate, so on CUDA cores those kernels
// are bound by the FP64 pipe at about a sixth of the memory bandwidth.  Here the basis is also
// held, written once per block when the block is made, as five FP16 planes of 11-bit integer
// digits (FP16 holds every integer up to 2^11 exactly):
//
//   v = 2^{e_c} sum_{p=0..4} a_p 2^{-11(p+1)},   a_p in [-1024, 1024]
//
// (2^{e_c - 1}: the power of two above the column's largest |v|, so the digits are v rounded to
// 55 bits of its largest entry).  The other operand -- the block Y, or the coefficient block
// with the basis column scales folded in -- is split for every product into eight planes of
// 7-bit digits b_q in [-64, 64] (56 bits), also FP16.  One MMA per basis digit plane p takes
// all eight digit planes q of the other operand at once (MMA N = 8 s, padded to a multiple of
// 16); every pair (p, q) accumulates integers in its own FP32 columns of tensor memory.  A
// pair's sum over 128 values of k is at most 2^10 * 2^6 * 128 = 2^23 in magnitude, so FP32
// holds it exactly; every 128 values of k the pairs of weight w = 11 p + 7 q <= 55 are added,
// as integers, into three int64 fixed-point words per output (w in [0, 20], [21, 41], [42, 55]).
// The result is the exact product of the rounded operands, rounded once to float64; the
// dropped pairs weigh less than 2^-58 (scale of v)(scale of the other operand) per term.
// (Ozaki scheme I: Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012; its tensor-core
// form: Mukunoki, Ozaki, Ogita, Imamura, ICCS 2020.)  Ten bytes per basis element: 11 of
// FP16's 16 bits carry digits, where 8-bit digits in BF16 carry 8 (seven planes, 14 bytes).
//
// Layouts (FP16 elements).  A tile holds T rows x 32 values of k in the canonical no-swizzle
// K-major layout of the tcgen05 shared-memory descriptor: 8-row x 16-byte core matrices, the
// four core matrices of an 8-row group adjacent.  The basis is stored twice, so that each
// kernel loads one chunk of a digit plane with one 1-D bulk copy (cp.async.bulk):
//   Gram layout   (tile rows = basis columns m, k = basis rows i): tile (i / 32, m / 128)
//   update layout (tile rows = basis rows i, k = basis columns m): tile (m / 32, i / 128)
// Each kernel reads 10 bytes per basis element instead of 8 (the second update of a step, whose
// coefficients are at rounding level, only the two leading planes: 4 bytes), and is bound by
// memory bandwidth instead of the FP64 pipe.
#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace sylv {

namespace {

constexpr int OB_PV = 5;          // digit planes of the basis
constexpr int OB_WV = 11;         // bits per basis digit
constexpr int OB_PY = 8;          // digit planes of the other operand
constexpr int OB_WY = 7;          // bits per digit of the other operand
constexpr int OB_WMAX = 55;       // pairs of weight 11 p + 7 q <= OB_WMAX are folded
constexpr int OB_TM = 128;        // MMA M: tile rows
constexpr int OB_KC = 32;         // k per chunk
constexpr int OB_FOLD = 4;        // chunks per fold (128 values of k)
constexpr int OB_STAGES = 4;      // chunks in flight for full 128-row tiles (more, smaller ones for narrow tiles)
constexpr int OB_MAXSTAGES = 16;
constexpr int OB_FOLD_THREADS = 128;  // warps 0-3 fold: TMEM lanes 0..127, one per tile row
constexpr int OB_THREADS = OB_FOLD_THREADS + 64;  // + warp 4: bulk copies, warp 5: MMAs
constexpr int OB_ATILE = OB_TM * OB_KC;  // FP16 elements of one basis digit tile (8 KB)
constexpr int OB_WAIT_ITERS = 1 << 20;
constexpr int OB_EXP_BAD = 1 << 20;      // exponent sentinel: a non-finite value

// Largest digit plane q of the other operand folded with basis plane p.
__host__ __device__ constexpr int ob_qmax(int p) {
  return (OB_WMAX - OB_WV * p) / OB_WY < OB_PY - 1 ? (OB_WMAX - OB_WV * p) / OB_WY : OB_PY - 1;
}
static_assert(OB_WV * (OB_PV - 1) <= OB_WMAX, "every basis plane meets at least one digit of the other operand");
static_assert((1 << (OB_WV - 1)) * (1 << (OB_WY - 1)) * (OB_FOLD * OB_KC) <= (1 << 23),
              "a fold period's pair sums stay exact in FP32");

template <int S>
struct ObShape {
  static constexpr int NP = (OB_PY * S + 15) / 16 * 16;  // MMA N: digit columns of the other operand
  static constexpr int BTILE = NP * OB_KC;               // FP16 elements of one of its tiles
  static constexpr int NBUF = 2 * OB_PV * NP <= 512 ? 2 : 1;  // accumulator buffers
  static constexpr int TMEM_COLS = NBUF * OB_PV * NP <= 256 ? 256 : 512;
  static constexpr uint32_t ABYTES = OB_ATILE * 2;
  static constexpr uint32_t BBYTES = BTILE * 2;
  static constexpr size_t STAGE = (size_t)OB_PV * ABYTES + BBYTES;
  static constexpr size_t REGION = OB_STAGES * STAGE;  // stage slots
  // + 8 KB: an MMA reads all 128 rows of a plane's tile, past a narrow slot's end
  static constexpr size_t SMEM = REGION + 8192 + 1024 + 512;
  // a 32-column TMEM load of the last plane of the last buffer stays inside the allocation
  static_assert((NBUF - 1) * OB_PV * NP + (OB_PV - 1) * NP + (((ob_qmax(OB_PV - 1) + 1) * S + 31) / 32) * 32 <=
                    TMEM_COLS, "tensor-memory loads stay in the allocation");
};

__device__ __forceinline__ uint32_t ob_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory descriptor, no swizzle: LBO 128 bytes (core matrices adjacent in k),
// SBO 512 bytes (8-row groups), descriptor version of this architecture family.
__device__ __forceinline__ uint64_t ob_sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: D FP32, A and B FP16 (type field 0), both K-major, M x N.
constexpr uint32_t ob_idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Offset of element (row i, k) inside a T x 32 tile.
__device__ __forceinline__ int ob_cm(int i, int k) {
  return (((i >> 3) * 4 + (k >> 3)) << 6) + ((i & 7) << 3) + (k & 7);
}

// e = 2 + floor(log2 m) for the IEEE bits m of a non-negative double (0 for zero or
// subnormal, OB_EXP_BAD for a non-finite value): every |x| <= m satisfies |x| < 2^{e-1}, one
// bit of headroom that keeps the leading digit within the range of the others.
__device__ __forceinline__ int ob_exponent(unsigned long long m) {
  if (m >= 0x7FF0000000000000ull) return OB_EXP_BAD;
  if (m < 0x0010000000000000ull) return 0;
  return (int)(m >> 52) - 1023 + 2;
}

// The D digits of W bits of x 2^sc on the scale 2^e (|x 2^sc| < 2^{e-1}): with B = D W,
// N = round(x 2^{sc+B-e}) (ties away from zero; |N| <= 2^{B-1}), sliced from the top with
// rounding to nearest, so that x 2^sc = 2^e sum_p d_p 2^{-W(p+1)} up to 2^{e-B-1}, every d_p
// in [-2^{W-1}, 2^{W-1}].  Integer operations only (the FP64 pipe is narrow on this GPU); zero
// and subnormal x give zero digits.
template <int D, int W>
__device__ __forceinline__ void ob_digits(double x, int sc, int e, int (&d)[D]) {
  constexpr int B = D * W;
  static_assert(B >= 54 && B <= 56, "the digits carry a float64 significand");
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  long long N = 0;
  if (ex != 0 && ex != 0x7FF && e != OB_EXP_BAD) {
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = ex - 1075 + sc + B - e;  // N = mant 2^sh; |x 2^sc| < 2^{e-1} gives sh <= B - 54
    unsigned long long u;
    if (sh >= 0)
      u = mant << sh;
    else if (sh < -54)
      u = 0;
    else
      u = (mant + (1ull << (-sh - 1))) >> (-sh);
    N = (b >> 63) ? -(long long)u : (long long)u;
  }
#pragma unroll
  for (int p = 0; p < D - 1; ++p) {
    const int s = W * (D - 1 - p);
    const long long dp = (N + (1ll << (s - 1))) >> s;
    N -= dp << s;
    d[p] = (int)dp;
  }
  d[D - 1] = (int)N;
}

__device__ __forceinline__ __half ob_h(int d) { return __int2half_rn(d); }  // |d| <= 1024: exact

// Digits of the new basis block (columns col0 .. col0 + S - 1, row-major n x S) into both
// layouts, and its column exponents into vexp.  One thread per basis row.
template <int S>
__global__ void __launch_bounds__(NT) ob_vsplit_kernel(const DevState* st, int64_t n, const double* __restrict__ Vb,
                                                       int col0, const unsigned long long* __restrict__ mx,
                                                       int* __restrict__ vexp, __half* __restrict__ G,
                                                       __half* __restrict__ U, int64_t plane, int MT, int IT) {
  if (stopped(st)) return;
  const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
  int e[S];
#pragma unroll
  for (int t = 0; t < S; ++t) e[t] = ob_exponent(mx[t]);
  if (i == 0)
    for (int t = 0; t < S; ++t) vexp[col0 + t] = e[t];
  if (i >= n) return;
#pragma unroll
  for (int t = 0; t < S; ++t) {
    int d[OB_PV];
    ob_digits<OB_PV, OB_WV>(Vb[i * S + t], 0, e[t], d);
    const int m = col0 + t;
    const int64_t og = ((i >> 5) * MT + (m >> 7)) * OB_ATILE + ob_cm(m & 127, (int)(i & 31));
    const int64_t ou = ((int64_t)(m >> 5) * IT + (i >> 7)) * OB_ATILE + ob_cm((int)(i & 127), m & 31);
#pragma unroll
    for (int p = 0; p < OB_PV; ++p) {
      G[p * plane + og] = ob_h(d[p]);
      U[p * plane + ou] = ob_h(d[p]);
    }
  }
}

// Digits of the block Y (n x S, row stride ldy) as the Gram's other operand: digit column
// q S + t of row (k =) i; exponents into ey.  Thread per (8 consecutive rows, column t): the 8
// rows' digits of a plane are one 16-byte core-matrix row, stored at once.  Rows from n up to
// the next multiple of 32 (the rest of the Gram's last 32-row chunk) get zero digits, so the
// operand never depends on what the buffer held before.
template <int S>
__global__ void __launch_bounds__(NT) ob_ysplit_kernel(const DevState* st, int64_t n, const double* __restrict__ Y,
                                                       int64_t ldy, const unsigned long long* __restrict__ mx,
                                                       int* __restrict__ ey, __half* __restrict__ YB) {
  if (stopped(st)) return;
  constexpr int NP = ObShape<S>::NP;
  const int64_t tid = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (tid < S) ey[tid] = ob_exponent(mx[tid]);
  const int64_t g = tid / S;
  const int t = (int)(tid - g * S);
  const int64_t i0 = g * 8;
  if (i0 >= (n + 31) / 32 * 32) return;
  const int e = ob_exponent(mx[t]);
  int d[OB_PY][8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    int dj[OB_PY];
    const double x = i0 + j < n ? Y[(i0 + j) * ldy + t] : 0.0;
    ob_digits<OB_PY, OB_WY>(x, 0, e, dj);
#pragma unroll
    for (int q = 0; q < OB_PY; ++q) d[q][j] = dj[q];
  }
  const int64_t base = (i0 >> 5) * (int64_t)(NP * OB_KC);
#pragma unroll
  for (int q = 0; q < OB_PY; ++q) {
    __align__(16) __half v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = ob_h(d[q][j]);
    *reinterpret_cast<uint4*>(YB + base + ob_cm(q * S + t, (int)(i0 & 31))) = *reinterpret_cast<const uint4*>(v);
  }
}

template <int S>
__device__ __forceinline__ void ob_hsplit_body(int js, const double* __restrict__ Hc, const int* __restrict__ vexp,
                                               int* __restrict__ eh, __half* __restrict__ HB,
                                               unsigned long long* __restrict__ mx) {
  if (threadIdx.x < 16) mx[threadIdx.x] = 0;
  constexpr int NP = ObShape<S>::NP;
  __shared__ long long kmax[NT / 32][S];
  __shared__ int esh[S];
  long long km[S];
#pragma unroll
  for (int t = 0; t < S; ++t) km[t] = LLONG_MIN;
  int bad = 0;
  for (int m = threadIdx.x; m < js; m += NT) {
    const int sc = vexp[m];
    if (sc == OB_EXP_BAD) bad = 1;
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const unsigned long long b =
          (unsigned long long)__double_as_longlong(__ldcg(Hc + (int64_t)m * S + t)) & 0x7FFFFFFFFFFFFFFFull;
      const int ex = (int)(b >> 52);
      if (ex == 0x7FF) bad = 1;
      else if (ex != 0 && sc != OB_EXP_BAD) km[t] = max(km[t], (long long)b + ((long long)sc << 52));
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < S; ++t) {
    long long v = km[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (l == 0) kmax[w][t] = v;
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x < S) {
    long long v = LLONG_MIN;
    for (int q = 0; q < NT / 32; ++q) v = max(v, kmax[q][threadIdx.x]);
    const int e = bad ? OB_EXP_BAD : (v == LLONG_MIN ? 0 : (int)(v >> 52) - 1023 + 2);
    esh[threadIdx.x] = e;
    eh[threadIdx.x] = e;
  }
  __syncthreads();
  const int kpad = (js + OB_KC - 1) / OB_KC * OB_KC;
  for (int m = threadIdx.x; m < kpad; m += NT) {
    const int sc = m < js ? vexp[m] : 0;
    const int64_t base = (int64_t)(m >> 5) * (NP * OB_KC);
#pragma unroll
    for (int t = 0; t < S; ++t) {
      int d[OB_PY];
      const double x = (m < js && sc != OB_EXP_BAD) ? __ldcg(Hc + (int64_t)m * S + t) : 0.0;
      ob_digits<OB_PY, OB_WY>(x, sc, esh[t], d);
#pragma unroll
      for (int q = 0; q < OB_PY; ++q) HB[base + ob_cm(q * S + t, m & 31)] = ob_h(d[q]);
    }
  }
}

// Digits of the coefficient block H'(m, t) = 2^{vexp[m]} Hc[m S + t] (m < js; zero up to the
// next multiple of 32) as the update's other operand, exponents into eh.  One CTA: the column
// maxima of H' come from integer keys bits(|Hc|) + vexp 2^52, which order like the values.
// Also zeroes the column maxima mx[0, 16): the ones of the update's result (the next Gram's Y)
// and of the block that CholQR will scale are combined into them from zero.
template <int S>
__global__ void __launch_bounds__(NT) ob_hsplit_kernel(const DevState* st, int js, const double* __restrict__ Hc,
                                                       const int* __restrict__ vexp, int* __restrict__ eh,
                                                       __half* __restrict__ HB, unsigned long long* __restrict__ mx) {
  if (stopped(st)) return;
  ob_hsplit_body<S>(js, Hc, vexp, eh, HB, mx);
}

// The BCGS2 coefficient block of one pass in one launch: H_{1:j,j} (+)= the sum of the Gram
// partials (partial[c E + e], E = nb S S, c < ncta, summed in a fixed order), also into Hc
// (js x S row-major), then the last CTA to finish (ticket) writes Hc's digits for the update
// (ob_hsplit_body).  256 threads: 8 outputs x 32 partial groups per CTA.
constexpr int OB_RED_E = 8, OB_RED_G = 32;
template <int S>
__global__ void __launch_bounds__(NT) ob_reduce_hsplit_kernel(DevState* st, const double* __restrict__ partial,
                                                              int ncta, int nb, double* __restrict__ H, int64_t ldh,
                                                              int64_t row0, int64_t col0, double* __restrict__ Hc,
                                                              int add, unsigned int* ticket, const int* __restrict__ vexp,
                                                              int* __restrict__ eh, __half* __restrict__ HB,
                                                              unsigned long long* __restrict__ mx) {
  if (stopped(st)) return;
  __shared__ double part[OB_RED_G][OB_RED_E];
  __shared__ int last_sh;
  const int E = nb * S * S;
  const int el = threadIdx.x % OB_RED_E, g = threadIdx.x / OB_RED_E;
  const int e = blockIdx.x * OB_RED_E + el;
  double v0 = 0.0, v1 = 0.0;
  if (e < E) {
    int c = g;
    for (; c + OB_RED_G < ncta; c += 2 * OB_RED_G) {
      v0 += partial[(int64_t)c * E + e];
      v1 += partial[(int64_t)(c + OB_RED_G) * E + e];
    }
    if (c < ncta) v0 += partial[(int64_t)c * E + e];
  }
  part[g][el] = v0 + v1;
  __syncthreads();
  if (g == 0 && e < E) {
    double vs = 0.0;
    for (int q = 0; q < OB_RED_G; ++q) vs += part[q][el];
    Hc[e] = vs;
    const int b = e / (S * S), r = e - b * S * S, u = r / S, t = r - u * S;
    double* h = H + (row0 + (int64_t)b * S + u) + (col0 + t) * ldh;
    *h = add ? (*h + vs) : vs;
  }
  if (!last_cta(ticket, &last_sh)) return;
  ob_hsplit_body<S>(nb * S, Hc, vexp, eh, HB, mx);
}

__device__ __forceinline__ bool ob_wait(uint32_t bar, uint32_t phase) {
  for (int it = 0; it < OB_WAIT_ITERS; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// v: an FP32 pair sum, an exact integer with |v| <= 2^23 (at most 128 products of a basis
// digit in [-1024, 1024] and one in [-64, 64]); the conversion is exact.
__device__ __forceinline__ long long ob_int(uint32_t r) { return (long long)__float2int_rn(__uint_as_float(r)); }

__device__ __forceinline__ double ob_pow2(int x) {  // 2^x as a float64 (0 or inf outside the normal range)
  return x < -1022 ? 0.0 : (x > 1023 ? __longlong_as_double(0x7FF0000000000000ll)
                                     : __longlong_as_double((long long)(x + 1023) << 52));
}

// 2^sc (w0 2^-38 + w1 2^-59 + w2 2^-73), the three fixed-point words of a fold, rounded once
// to float64 (nearest, ties to even) with integer operations: the words are aligned into one
// 128-bit integer W of unit 2^-73 (|W| < 2^98), whose leading 53 bits give the significand.
// GB300's FP64 pipe is narrow, and this runs once per output in the epilogues.  A result
// outside the normal float64 range takes the float64 formula (rounded more than once).
__device__ __forceinline__ double ob_fixed_to_double(long long w0, long long w1, long long w2, int sc) {
  const __int128 W = ((__int128)w0 << 35) + ((__int128)w1 << 14) + (__int128)w2;
  if (W == 0) return 0.0;
  const unsigned long long sign = W < 0 ? 1ull : 0ull;
  const unsigned __int128 M = sign ? (unsigned __int128)(-W) : (unsigned __int128)W;
  const unsigned long long mh = (unsigned long long)(M >> 64), ml = (unsigned long long)M;
  int b = mh ? 127 - __clzll((long long)mh) : 63 - __clzll((long long)ml);  // leading bit of M
  unsigned long long keep;
  if (b <= 52) {
    keep = ml << (52 - b);
  } else {
    const int sh = b - 52;
    const unsigned __int128 q = M >> sh;
    const unsigned __int128 rem = M - (q << sh);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    keep = (unsigned long long)q;
    if (rem > half || (rem == half && (keep & 1ull))) ++keep;
    if (keep >> 53) {
      keep >>= 1;
      ++b;
    }
  }
  const int ex = b + sc - 73 + 1023;  // biased exponent of (keep 2^-52) 2^{b + sc - 73}
  if (ex <= 0 || ex >= 2047)
    return fma((double)w0, 0x1p-38, fma((double)w1, 0x1p-59, (double)w2 * 0x1p-73)) * ob_pow2(sc / 2) *
           ob_pow2(sc - sc / 2);
  return __longlong_as_double((long long)((sign << 63) | ((unsigned long long)ex << 52) | (keep & 0xFFFFFFFFFFFFFull)));
}

struct ObArgs {
  DevState* st;
  const __half* A;         // basis digit planes (Gram or update layout)
  int64_t plane;           // elements per plane
  int MT;                  // tiles per chunk row of that layout (Gram: Rp / 128, update: np / 128)
  const __half* B;         // digits of the other operand, one NP x 32 tile per chunk
  int64_t n;               // basis rows
  int js;                  // basis columns in use
  int cps;                 // Gram: chunks per k split (blockIdx.y)
  const int* ea;           // Gram: exponents of the basis columns
  const int* eb;           // exponents of the other operand's columns
  double* out;             // Gram: partials [split][m S + t]; update: Y (row-major n x S)
  double* self;            // update: per-CTA partial Y^T Y of the result (nullptr: none)
  unsigned long long* ymax;  // update: column maxima of |result| as IEEE bits (nullptr: none)
  int planes;              // basis digit planes used (the leading ones; OB_PV: all)
  int64_t ldy;             // update: row stride of Y (S for a block of its own)
  int add;                 // update: Y += V H instead of Y -= V H
};

// GRAM: CTA (m tile, k split) writes the partial V^T Y of its rows.  Update: CTA c takes
// row tiles c, c + grid, ... and subtracts V H from those rows of Y.  Warp 4 (one lane) issues
// the bulk copies into the stage slots as they free up; warp 5 (one lane) issues the MMAs as the
// chunks land; warps 0-3 fold the tensor memory once per OB_FOLD chunks (a fold period) and
// write the results.  With two accumulator buffers the MMAs of a period run while the previous
// period is folded.  A wait that gives up sets the solve status to ST_WAIT_TIMEOUT.
template <int S, bool GRAM>
__global__ void __launch_bounds__(OB_THREADS, 1) ob_kernel(ObArgs a) {
  using Sh = ObShape<S>;
  constexpr int NP = Sh::NP;
  constexpr int NBUF = Sh::NBUF;
  if (stopped(a.st)) return;
  extern __shared__ __align__(1024) unsigned char ob_smem[];
  unsigned char* base = (unsigned char*)(((uintptr_t)ob_smem + 1023) & ~(uintptr_t)1023);
  // barriers: full[MAXSTAGES], empty[MAXSTAGES] (copies / MMAs of a stage), accf[2] (a
  // buffer's period is accumulated), acce[2] (a buffer is folded), done (MMAs of a failed run)
  uint64_t* bars = (uint64_t*)(base + Sh::REGION + 8192);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * OB_MAXSTAGES + 5);
  __shared__ double shred[4 * S * S];
  __shared__ unsigned long long smx[4][S];
  __shared__ int fail_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  int ntiles, nch, c0 = 0, rg = OB_TM / 8;
  const int mt = (int)blockIdx.x;
  if (GRAM) {
    // every split of every tile has the same number of chunks: the MMAs of a chunk cost the
    // same for a narrow tile, and they bound a narrow tile's chunk, not its bytes
    const int kcn = (int)((a.n + OB_KC - 1) / OB_KC);
    c0 = (int)blockIdx.y * a.cps;
    nch = max(0, min(a.cps, kcn - c0));
    ntiles = 1;
    rg = min(OB_TM / 8, (a.js - mt * OB_TM + 7) / 8);  // 8-row groups holding basis columns
  } else {
    const int it = (int)((a.n + OB_TM - 1) / OB_TM);
    ntiles = (int)blockIdx.x < it ? (it - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    nch = (a.js + OB_KC - 1) / OB_KC;
  }
  const uint32_t abytes = (uint32_t)rg * 512;  // per digit plane and chunk: the tile's row groups
  // A stage holds G chunks: every stage costs a barrier round trip between the copy and MMA
  // warps, and stages of 16 KB or less (the two-plane update, narrow Gram tiles) were measured
  // to cap a CTA near 36 GB/s however many are in flight; 32 KB and more reach the copy rate.
  const uint32_t cbytes = a.planes * abytes + Sh::BBYTES;  // one chunk: basis planes, then the other operand
  const int G = a.planes * abytes <= 16384u ? 2 : 1;
  const int nit = (nch + G - 1) / G;  // stages per tile
  const int NI = ntiles * nit;
  const int npt = (nch + OB_FOLD - 1) / OB_FOLD;  // fold periods per tile
  const int NF = ntiles * npt;
  // stage slots: a narrow tile (Gram, few basis columns) or fewer digit planes get more of them,
  // so that about the same number of bytes stays in flight
  const uint32_t slot = (uint32_t)G * cbytes;
  const int ns = min(OB_MAXSTAGES, (int)(Sh::REGION / slot));

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(ob_smem_u32(tmem_slot)),
                 "r"(Sh::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  const uint32_t bfull = ob_smem_u32(bars), bempty = ob_smem_u32(bars + OB_MAXSTAGES),
                 baccf = ob_smem_u32(bars + 2 * OB_MAXSTAGES), bacce = ob_smem_u32(bars + 2 * OB_MAXSTAGES + 2),
                 bdone = ob_smem_u32(bars + 2 * OB_MAXSTAGES + 4);
  if (tid == 0) {
    for (int i = 0; i < 2 * OB_MAXSTAGES + 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ob_smem_u32(bars + i)));
    for (int i = 0; i < 2; ++i)  // every fold thread arrives
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bacce + 8 * i), "r"(OB_FOLD_THREADS));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bdone));
    asm volatile("fence.mbarrier_init.release.cluster;");
    fail_sh = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  __shared__ int issued_sh, consumed_sh;  // items whose copies were issued / whose MMAs were issued

  if (warp == OB_FOLD_THREADS / 32) {
    // ---------------------------------------------------------------- bulk copies
    if (lane == 0) {
      bool ok = true;
      int i = 0;
      for (; i < NI; ++i) {
        const int stg = i % ns;
        // the stage is free once the MMAs of its previous chunks are done
        if (i >= ns && !ob_wait(bempty + 8 * stg, (uint32_t)(i / ns - 1) & 1u)) {
          ok = false;
          break;
        }
        const int tile = i / nit, cfirst = (i - tile * nit) * G, cn = min(G, nch - cfirst);
        const uint32_t bar = bfull + 8 * stg;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)cn * cbytes)
                     : "memory");
        for (int u = 0; u < cn; ++u) {
          const int c = cfirst + u;
          unsigned char* sa = base + stg * slot + u * cbytes;
          unsigned char* sb = sa + a.planes * abytes;
          const __half* ga;
          const __half* gb;
          if (GRAM) {
            const int kc = c0 + c;
            ga = a.A + ((int64_t)kc * a.MT + mt) * OB_ATILE;
            gb = a.B + (int64_t)kc * Sh::BTILE;
          } else {
            const int it = (int)blockIdx.x + tile * (int)gridDim.x;
            ga = a.A + ((int64_t)c * a.MT + it) * OB_ATILE;
            gb = a.B + (int64_t)c * Sh::BTILE;
          }
#pragma unroll 1
          for (int p = 0; p < a.planes; ++p)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             ob_smem_u32(sa + p * abytes)),
                         "l"(ga + p * a.plane), "r"(abytes), "r"(bar)
                         : "memory");
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                           ob_smem_u32(sb)),
                       "l"(gb), "r"(Sh::BBYTES), "r"(bar)
                       : "memory");
        }
      }
      issued_sh = i;
      if (!ok) fail_sh = 1;
    }
    __syncwarp();
  } else if (warp == OB_FOLD_THREADS / 32 + 1) {
    // ---------------------------------------------------------------- MMAs
    if (lane == 0) {
      const uint32_t id = ob_idesc(OB_TM, NP);
      bool ok = true;
      int i = 0;
      for (; i < NI; ++i) {
        const int tile = i / nit, cfirst = (i - tile * nit) * G, cn = min(G, nch - cfirst);
        const int stg = i % ns;
        if (!ob_wait(bfull + 8 * stg, (uint32_t)(i / ns) & 1u)) ok = false;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int u = 0; u < cn && ok; ++u) {
          const int c = cfirst + u;
          const int f = tile * npt + c / OB_FOLD, buf = f % NBUF;
          const bool first = (c % OB_FOLD) == 0;
          const bool last = (c % OB_FOLD) == OB_FOLD - 1 || c == nch - 1;
          // the accumulator buffer is free once the fold of its previous period is done
          if (first && f >= NBUF && !ob_wait(bacce + 8 * buf, (uint32_t)(f / NBUF - 1) & 1u)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t sa = ob_smem_u32(base + stg * slot + u * cbytes), sb = sa + a.planes * abytes;
          const uint32_t dbase = tmem + (uint32_t)(buf * OB_PV * NP);
#pragma unroll 1
          for (int p = 0; p < a.planes; ++p) {
#pragma unroll
            for (int ks = 0; ks < OB_KC / 16; ++ks) {
              const uint64_t da = ob_sdesc(sa + p * abytes + ks * 256);
              const uint64_t db = ob_sdesc(sb + ks * 256);
              const uint32_t accf = (first && ks == 0) ? 0u : 1u;  // a period starts each plane afresh
              asm volatile(
                  "{\n .reg .pred pa;\n setp.ne.b32 pa, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}\n" ::"r"(dbase + (uint32_t)(p * NP)),
                  "l"(da), "l"(db), "r"(id), "r"(accf)
                  : "memory");
            }
          }
          if (last)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             baccf + 8 * buf)
                         : "memory");
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         bempty + 8 * stg)
                     : "memory");
      }
      consumed_sh = i;
      if (!ok) fail_sh = 1;
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- folds and results
    // pair sums of weight w = 11 p + 7 q (unit 2^{-18-w}) in three words: w in [0, 20] (unit
    // 2^-38), [21, 41] (2^-59), [42, 55] (2^-73)
    long long w0[S], w1[S], w2[S];
    double acc[S][S];               // update: partial Y^T Y
    unsigned long long ym[S];       // update: column maxima of |result|
#pragma unroll
    for (int t = 0; t < S; ++t) {
      ym[t] = 0;
      w0[t] = w1[t] = w2[t] = 0;
#pragma unroll
      for (int u = 0; u < S; ++u) acc[u][t] = 0.0;
    }
    bool ok = true;
    for (int f = 0; f < NF; ++f) {
      const int buf = f % NBUF;
      // update: the last period of a tile; its rows of Y are loaded before the wait, so that
      // their latency passes while the MMAs finish
      const bool tile_end = !GRAM && f % npt == npt - 1;
      const int64_t row = (int64_t)((int)blockIdx.x + (f / npt) * (int)gridDim.x) * OB_TM + tid;
      double yold[S];
      if (tile_end && row < a.n) {
#pragma unroll
        for (int t = 0; t < S; ++t) yold[t] = a.out[row * a.ldy + t];
      }
      if (!ob_wait(baccf + 8 * buf, (uint32_t)(f / NBUF) & 1u)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * OB_PV * NP);
#pragma unroll
      for (int p = 0; p < OB_PV; ++p) {
        constexpr int NCMAX = OB_PY * S;
#pragma unroll
        for (int cb = 0; cb < NCMAX; cb += 32) {
          if (p < a.planes && cb < (ob_qmax(p) + 1) * S) {
            uint32_t r[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(tbase + (uint32_t)(p * NP + cb)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int col = cb + j, q = col / S, t = col % S, w = OB_WV * p + OB_WY * q;
              if (q <= ob_qmax(p)) {
                const long long v = ob_int(r[j]);
                if (w <= 20)
                  w0[t] += v * (1ll << (20 - w));
                else if (w <= 41)
                  w1[t] += v * (1ll << (41 - w));
                else
                  w2[t] += v * (1ll << (55 - w));
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bacce + 8 * buf) : "memory");
      if (tile_end) {  // the tile is complete: Y -= V H on its rows
        if (row < a.n) {
          double y[S];
#pragma unroll
          for (int t = 0; t < S; ++t) {
            const int fe = a.eb[t];
            const double v = fe == OB_EXP_BAD ? __longlong_as_double(0x7FF8000000000000ll)
                                              : ob_fixed_to_double(w0[t], w1[t], w2[t], fe);
            y[t] = a.add ? yold[t] + v : yold[t] - v;
          }
#pragma unroll
          for (int t = 0; t < S; ++t) {
            a.out[row * a.ldy + t] = y[t];
            ym[t] = max(ym[t], (unsigned long long)__double_as_longlong(fabs(y[t])));
          }
          if (a.self) {  // the upper triangle (the partial is symmetric)
#pragma unroll
            for (int u = 0; u < S; ++u)
#pragma unroll
              for (int t = u; t < S; ++t) acc[u][t] += y[u] * y[t];
          }
        }
#pragma unroll
        for (int t = 0; t < S; ++t) w0[t] = w1[t] = w2[t] = 0;
      }
    }
    if (!ok) fail_sh = 1;
    if (ok && GRAM) {
      const int m = mt * OB_TM + tid;
      if (m < a.js) {
        const int e = a.ea[m];
        double* o = a.out + (int64_t)blockIdx.y * ((int64_t)a.js * S) + (int64_t)m * S;
#pragma unroll
        for (int t = 0; t < S; ++t) {
          const int fe = a.eb[t];
          const double v = (e == OB_EXP_BAD || fe == OB_EXP_BAD) ? __longlong_as_double(0x7FF8000000000000ll)
                                                                 : ob_fixed_to_double(w0[t], w1[t], w2[t], e + fe);
          o[t] = v;
        }
      }
    }
    if (!GRAM && a.ymax) {
#pragma unroll
      for (int t = 0; t < S; ++t) {
        unsigned long long v = ym[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) smx[warp][t] = v;
      }
    }
    if (!GRAM && a.self) {
#pragma unroll
      for (int u = 0; u < S; ++u)
#pragma unroll
        for (int t = 0; t < S; ++t) {
          double v = u <= t ? acc[u][t] : acc[t][u];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) shred[warp * S * S + u * S + t] = v;
        }
    }
  }
  __syncthreads();
  if (fail_sh) {
    if (tid == OB_FOLD_THREADS) {
      a.st->breakdown_where = GRAM ? 210 : 211;
      atomicExch(&a.st->status, (int)ST_WAIT_TIMEOUT);
      // copies still in flight land in shared memory: wait for them (bounded)
      for (int j = consumed_sh; j < issued_sh; ++j) ob_wait(bfull + 8 * (j % ns), (uint32_t)(j / ns) & 1u);
    } else if (tid == OB_FOLD_THREADS + 32) {  // the MMAs this thread issued (bounded)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bdone)
                   : "memory");
      ob_wait(bdone, 0);
    }
  } else {
    if (!GRAM && a.self && tid < S * S) {
      double v = 0.0;
      for (int q = 0; q < 4; ++q) v += shred[q * S * S + tid];
      a.self[(int64_t)blockIdx.x * S * S + tid] = v;
    }
    if (!GRAM && a.ymax && tid < S) {
      unsigned long long v = 0;
      for (int q = 0; q < 4; ++q) v = max(v, smx[q][tid]);
      if (v) atomicMax(a.ymax + tid, v);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::TMEM_COLS));
}

// Column maxima of |V| over the nb blocks of a basis (block b: n x S row-major at V + b bstride,
// element T) as IEEE bits of the float64 value into mx[b S + t] (zeroed beforehand).  Grid: (row
// chunks, blocks).
template <int S, typename T>
__global__ void __launch_bounds__(NT) ob_colmax_blocks_kernel(int64_t n, const T* __restrict__ V, int64_t bstride,
                                                              unsigned long long* __restrict__ mx) {
  __shared__ unsigned long long sm[S];
  if (threadIdx.x < S) sm[threadIdx.x] = 0;
  __syncthreads();
  const T* Vb = V + (int64_t)blockIdx.y * bstride;
  unsigned long long m[S];
#pragma unroll
  for (int t = 0; t < S; ++t) m[t] = 0;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT)
#pragma unroll
    for (int t = 0; t < S; ++t)
      m[t] = max(m[t], (unsigned long long)__double_as_longlong((double)Vb[i * S + t]) & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
  for (int t = 0; t < S; ++t) {
    unsigned long long v = m[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(&sm[t], v);
  }
  __syncthreads();
  if (threadIdx.x < S && sm[threadIdx.x]) atomicMax(mx + (int64_t)blockIdx.y * S + threadIdx.x, sm[threadIdx.x]);
}

// Digits of all nb blocks of a basis (element T, float64 or float32: both exact in 53 bits)
// into both layouts, and the column exponents into vexp; the column maxima in mx[b S + t].
// Thread per (row, block): grid (row chunks, blocks).
template <int S, typename T>
__global__ void __launch_bounds__(NT) ob_vsplit_blocks_kernel(int64_t n, const T* __restrict__ V, int64_t bstride,
                                                              const unsigned long long* __restrict__ mx,
                                                              int* __restrict__ vexp, __half* __restrict__ G,
                                                              __half* __restrict__ U, int64_t plane, int MT, int IT) {
  const int b = (int)blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
  int e[S];
#pragma unroll
  for (int t = 0; t < S; ++t) e[t] = ob_exponent(mx[(int64_t)b * S + t]);
  if (i == 0)
    for (int t = 0; t < S; ++t) vexp[b * S + t] = e[t];
  if (i >= n) return;
  const T* Vb = V + (int64_t)b * bstride;
#pragma unroll
  for (int t = 0; t < S; ++t) {
    int d[OB_PV];
    ob_digits<OB_PV, OB_WV>((double)Vb[i * S + t], 0, e[t], d);
    const int m = b * S + t;
    const int64_t og = ((i >> 5) * MT + (m >> 7)) * OB_ATILE + ob_cm(m & 127, (int)(i & 31));
    const int64_t ou = ((int64_t)(m >> 5) * IT + (i >> 7)) * OB_ATILE + ob_cm((int)(i & 127), m & 31);
#pragma unroll
    for (int p = 0; p < OB_PV; ++p) {
      G[p * plane + og] = ob_h(d[p]);
      U[p * plane + ou] = ob_h(d[p]);
    }
  }
}

// Column maxima of |Y| (n x S, row stride ldy) as IEEE bits (non-negative doubles order like
// their bit patterns), combined into mx (zeroed beforehand) with atomicMax: the true-residual
// certificate's blocks, whose producers do not record them.
template <int S>
__global__ void __launch_bounds__(NT) ob_colmax_kernel(int64_t n, const double* __restrict__ Y, int64_t ldy,
                                                       unsigned long long* __restrict__ mx) {
  __shared__ unsigned long long sm[S];
  if (threadIdx.x < S) sm[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long m[S];
#pragma unroll
  for (int t = 0; t < S; ++t) m[t] = 0;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT)
#pragma unroll
    for (int t = 0; t < S; ++t)
      m[t] = max(m[t], (unsigned long long)__double_as_longlong(Y[i * ldy + t]) & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
  for (int t = 0; t < S; ++t) {
    unsigned long long v = m[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(&sm[t], v);
  }
  __syncthreads();
  if (threadIdx.x < S && sm[threadIdx.x]) atomicMax(mx + threadIdx.x, sm[threadIdx.x]);
}

// P[m ldp + col0 + t] = the sum over the ks splits of partial[z][m S + t] (m < js), in split order.
template <int S>
__global__ void __launch_bounds__(NT) ob_sum_splits_kernel(int ks, int js, const double* __restrict__ partial,
                                                           double* __restrict__ P, int64_t ldp, int col0) {
  const int idx = blockIdx.x * NT + threadIdx.x;
  if (idx >= js * S) return;
  double v = 0.0;
  for (int z = 0; z < ks; ++z) v += partial[(int64_t)z * js * S + idx];
  P[(int64_t)(idx / S) * ldp + col0 + idx % S] = v;
}

int ob_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
}

int ob_np(int64_t n) { return (int)((n + OB_TM - 1) / OB_TM * OB_TM); }
int ob_rp(int R) { return (R + OB_TM - 1) / OB_TM * OB_TM; }
int ob_NP(int s) { return (OB_PY * s + 15) / 16 * 16; }

template <typename F>
bool ob_for_each_kernel(F f) {
  bool ok = true;
#define OB_CASE(SV) \
  ok = ok && f((const void*)ob_kernel<SV, true>, ObShape<SV>::SMEM) && f((const void*)ob_kernel<SV, false>, ObShape<SV>::SMEM);
  OB_CASE(1) OB_CASE(2) OB_CASE(3) OB_CASE(4) OB_CASE(5) OB_CASE(6) OB_CASE(7) OB_CASE(8)
#undef OB_CASE
  return ok;
}

}  // namespace

size_t ob_side_bytes(int64_t n, int R, int s) {
  const size_t np = (size_t)ob_np(n), rp = (size_t)ob_rp(R), NPs = (size_t)ob_NP(s);
  return 256 + 2 * (size_t)OB_PV * np * rp * 2  // Gram and update layouts
         + np * NPs * 2 + rp * NPs * 2          // digits of Y and of the coefficient block
         + rp * sizeof(int) + 16 * sizeof(int)  // basis column exponents, ey, eh
         + 16 * sizeof(unsigned long long) + 1024;
}

void ob_carve(void* mem, int64_t n, int R, int s, ObSide& o) {
  const size_t np = (size_t)ob_np(n), rp = (size_t)ob_rp(R), NPs = (size_t)ob_NP(s);
  uintptr_t p = ((uintptr_t)mem + 255) & ~(uintptr_t)255;
  auto take = [&](size_t bytes) {
    void* q = (void*)p;
    p = (p + bytes + 255) & ~(uintptr_t)255;
    return q;
  };
  o.np = (int64_t)np;
  o.rp = (int)rp;
  o.plane = (int64_t)(np * rp);
  o.G = (uint16_t*)take((size_t)OB_PV * np * rp * 2);
  o.U = (uint16_t*)take((size_t)OB_PV * np * rp * 2);
  o.YB = (uint16_t*)take(np * NPs * 2);
  o.HB = (uint16_t*)take(rp * NPs * 2);
  o.vexp = (int*)take(rp * sizeof(int));
  o.ey = (int*)take(8 * sizeof(int));
  o.eh = (int*)take(8 * sizeof(int));
  o.mx = (unsigned long long*)take(16 * sizeof(unsigned long long));
}

bool ob_setup() {
  return ob_for_each_kernel([](const void* fn, size_t smem) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
  });
}

#define SYLV_OB_S_CASES(MACRO) MACRO(1) MACRO(2) MACRO(3) MACRO(4) MACRO(5) MACRO(6) MACRO(7) MACRO(8)

void launch_ob_split_basis(cudaStream_t strm, const DevState* st, int64_t n, int s, const double* Vb, int col0,
                           const ObSide& o) {
  if (n == 0) return;
  const unsigned gs = (unsigned)((n + NT - 1) / NT);
  __half* G = (__half*)o.G;
  __half* U = (__half*)o.U;
  const int MT = o.rp / OB_TM, IT = (int)(o.np / OB_TM);
#define CASE(SV)                                                                                           \
  case SV:                                                                                                 \
    ob_vsplit_kernel<SV><<<counted(gs), NT, 0, strm>>>(st, n, Vb, col0, o.mx, o.vexp, G, U, o.plane, MT, IT); \
    break;
  switch (s) { SYLV_OB_S_CASES(CASE) }
#undef CASE
}

int launch_ob_gram(cudaStream_t strm, DevState* st, int64_t n, int s, int js, const double* Y, const ObSide& o,
                   double* partial) {
  // digit split: a thread per (8 rows, column) up to the next multiple of 32 rows
  const unsigned gs = (unsigned)std::max<int64_t>(1, ((n + 31) / 32 * 4 * s + NT - 1) / NT);
  const int mtv = (js + OB_TM - 1) / OB_TM;
  const int kcn = (int)std::max<int64_t>(1, (n + OB_KC - 1) / OB_KC);
  int ks = std::max(1, std::min(kcn, ob_sms() / mtv));
  const int cps = (kcn + ks - 1) / ks;
  ks = (kcn + cps - 1) / cps;  // no empty split
  ObArgs a{};
  a.st = st;
  a.A = (const __half*)o.G;
  a.plane = o.plane;
  a.MT = o.rp / OB_TM;
  a.B = (const __half*)o.YB;
  a.n = n;
  a.js = js;
  a.cps = cps;
  a.ea = o.vexp;
  a.eb = o.ey;
  a.out = partial;
  a.self = nullptr;
  a.ymax = nullptr;
  a.planes = OB_PV;
  a.ldy = s;
  a.add = 0;
  const dim3 grid((unsigned)mtv, (unsigned)ks);
#define CASE(SV)                                                                                                 \
  case SV:                                                                                                       \
    ob_ysplit_kernel<SV><<<counted(gs), NT, 0, strm>>>(st, n, Y, SV, o.mx + 8, o.ey, (__half*)o.YB);                  \
    ob_kernel<SV, true><<<counted(grid), OB_THREADS, ObShape<SV>::SMEM, strm>>>(a);                              \
    break;
  switch (s) { SYLV_OB_S_CASES(CASE) }
#undef CASE
  return ks;
}

int launch_ob_update(cudaStream_t strm, DevState* st, int64_t n, int s, int js, const double* Hc, double* Y,
                     const ObSide& o, double* self_partial, bool ymax, int planes, bool split_done) {
  const int itn = (int)std::max<int64_t>(1, (n + OB_TM - 1) / OB_TM);
  const int grid = std::min(itn, ob_sms());
  ObArgs a{};
  a.st = st;
  a.A = (const __half*)o.U;
  a.plane = o.plane;
  a.MT = (int)(o.np / OB_TM);
  a.B = (const __half*)o.HB;
  a.n = n;
  a.js = js;
  a.cps = 0;
  a.ea = nullptr;
  a.eb = o.eh;
  a.out = Y;
  a.self = self_partial;
  a.ymax = ymax ? o.mx + 8 : nullptr;
  a.planes = std::max(1, std::min(OB_PV, planes));
  a.ldy = s;
  a.add = 0;
#define CASE(SV)                                                                                              \
  case SV:                                                                                                    \
    if (!split_done)                                                                                          \
      ob_hsplit_kernel<SV><<<counted(1), NT, 0, strm>>>(st, js, Hc, o.vexp, o.eh, (__half*)o.HB, o.mx);        \
    ob_kernel<SV, false><<<counted(grid), OB_THREADS, ObShape<SV>::SMEM, strm>>>(a);                          \
    break;
  switch (s) { SYLV_OB_S_CASES(CASE) }
#undef CASE
  return grid;
}

// ---------------------------------------------------------------- certificate products
size_t ob_cols_scratch_bytes(int64_t n_max, int R_max, int S) {
  const size_t np = (size_t)ob_np(n_max), rp = (size_t)ob_rp(R_max), NPs = (size_t)ob_NP(S);
  return 256 + np * NPs * 2 + rp * NPs * 2 + 16 * sizeof(int) + 16 * sizeof(unsigned long long) + 1024;
}

void ob_cols_carve(void* mem, int64_t n_max, int R_max, int S, ObSide& o) {
  const size_t np = (size_t)ob_np(n_max), rp = (size_t)ob_rp(R_max), NPs = (size_t)ob_NP(S);
  uintptr_t p = ((uintptr_t)mem + 255) & ~(uintptr_t)255;
  auto take = [&](size_t bytes) {
    void* q = (void*)p;
    p = (p + bytes + 255) & ~(uintptr_t)255;
    return q;
  };
  o.YB = (uint16_t*)take(np * NPs * 2);
  o.HB = (uint16_t*)take(rp * NPs * 2);
  o.ey = (int*)take(8 * sizeof(int));
  o.eh = (int*)take(8 * sizeof(int));
  o.mx = (unsigned long long*)take(16 * sizeof(unsigned long long));
}

int launch_ob_gram_cols(cudaStream_t strm, DevState* st, int64_t n, int s, int js, const double* Y, int64_t ldy,
                        const ObSide& o, double* partial, double* P, int64_t ldp, int col0) {
  if (js <= 0) return 0;
  // digit split: a thread per (8 rows, column) up to the next multiple of 32 rows
  const unsigned gs = (unsigned)std::max<int64_t>(1, ((n + 31) / 32 * 4 * s + NT - 1) / NT);
  const unsigned gm = (unsigned)std::min<int64_t>(std::max<int64_t>(1, (n + NT - 1) / NT), 2 * ob_sms());
  const int mtv = (js + OB_TM - 1) / OB_TM;
  const int kcn = (int)std::max<int64_t>(1, (n + OB_KC - 1) / OB_KC);
  int ks = std::max(1, std::min(kcn, ob_sms() / mtv));
  const int cps = (kcn + ks - 1) / ks;
  ks = (kcn + cps - 1) / cps;  // no empty split
  ObArgs a{};
  a.st = st;
  a.A = (const __half*)o.G;
  a.plane = o.plane;
  a.MT = o.rp / OB_TM;
  a.B = (const __half*)o.YB;
  a.n = n;
  a.js = js;
  a.cps = cps;
  a.ea = o.vexp;
  a.eb = o.ey;
  a.out = partial;
  a.planes = OB_PV;
  a.ldy = s;
  a.add = 0;
  const dim3 grid((unsigned)mtv, (unsigned)ks);
  const unsigned gr = (unsigned)(((int64_t)js * s + NT - 1) / NT);
  cudaMemsetAsync(o.mx + 8, 0, 8 * sizeof(unsigned long long), strm);
#define CASE(SV)                                                                                                 \
  case SV:                                                                                                       \
    ob_colmax_kernel<SV><<<counted(gm), NT, 0, strm>>>(n, Y, ldy, o.mx + 8);                                     \
    ob_ysplit_kernel<SV><<<counted(gs), NT, 0, strm>>>(st, n, Y, ldy, o.mx + 8, o.ey, (__half*)o.YB);            \
    ob_kernel<SV, true><<<counted(grid), OB_THREADS, ObShape<SV>::SMEM, strm>>>(a);                              \
    ob_sum_splits_kernel<SV><<<counted(gr), NT, 0, strm>>>(ks, js, partial, P, ldp, col0);                       \
    break;
  switch (s) { SYLV_OB_S_CASES(CASE) }
#undef CASE
  return ks;
}

void launch_ob_update_cols(cudaStream_t strm, DevState* st, int64_t n, int s, int js, const double* Hc, double* Z,
                           int64_t ldz, const ObSide& o) {
  if (js <= 0 || n == 0) return;
  const int itn = (int)std::max<int64_t>(1, (n + OB_TM - 1) / OB_TM);
  const int grid = std::min(itn, ob_sms());
  ObArgs a{};
  a.st = st;
  a.A = (const __half*)o.U;
  a.plane = o.plane;
  a.MT = (int)(o.np / OB_TM);
  a.B = (const __half*)o.HB;
  a.n = n;
  a.js = js;
  a.eb = o.eh;
  a.out = Z;
  a.self = nullptr;
  a.ymax = nullptr;
  a.planes = OB_PV;
  a.ldy = ldz;
  a.add = 1;
#define CASE(SV)                                                                                              \
  case SV:                                                                                                    \
    ob_hsplit_kernel<SV><<<counted(1), NT, 0, strm>>>(st, js, Hc, o.vexp, o.eh, (__half*)o.HB, o.mx);          \
    ob_kernel<SV, false><<<counted(grid), OB_THREADS, ObShape<SV>::SMEM, strm>>>(a);                          \
    break;
  switch (s) { SYLV_OB_S_CASES(CASE) }
#undef CASE
}

void launch_ob_split_bases(cudaStream_t strm, int64_t n, int s, int nb, const void* V, bool is_float, int64_t bstride,
                           unsigned long long* mx_all, const ObSide& o) {
  if (n == 0 || nb == 0) return;
  cudaMemsetAsync(mx_all, 0, (size_t)nb * s * sizeof(unsigned long long), strm);
  const unsigned gx = (unsigned)((n + NT - 1) / NT);
  const dim3 gm((unsigned)std::min<int64_t>(gx, 16), (unsigned)nb);
  const dim3 gs(gx, (unsigned)nb);
  __half* G = (__half*)o.G;
  __half* U = (__half*)o.U;
  const int MT = o.rp / OB_TM, IT = (int)(o.np / OB_TM);
#define CASE(SV)                                                                                                   \
  case SV:                                                                                                         \
    if (is_float) {                                                                                                \
      ob_colmax_blocks_kernel<SV, float><<<counted(gm), NT, 0, strm>>>(n, (const float*)V, bstride, mx_all);       \
      ob_vsplit_blocks_kernel<SV, float><<<counted(gs), NT, 0, strm>>>(n, (const float*)V, bstride, mx_all,        \
                                                                       o.vexp, G, U, o.plane, MT, IT);             \
    } else {                                                                                                       \
      ob_colmax_blocks_kernel<SV, double><<<counted(gm), NT, 0, strm>>>(n, (const double*)V, bstride, mx_all);     \
      ob_vsplit_blocks_kernel<SV, double><<<counted(gs), NT, 0, strm>>>(n, (const double*)V, bstride, mx_all,      \
                                                                        o.vexp, G, U, o.plane, MT, IT);            \
    }                                                                                                              \
    break;
  switch (s) { SYLV_OB_S_CASES(CASE) }
#undef CASE
}

void launch_ob_reduce_H(cudaStream_t strm, DevState* st, int side, const double* partial, int ncta, int nb, int s,
                        double* H, int64_t ldh, int64_t row0, int64_t col0, double* Hc, bool add, const ObSide& o) {
  const int E = nb * s * s;
  const unsigned grid = (unsigned)((E + OB_RED_E - 1) / OB_RED_E);
  unsigned int* ticket = &st->tickets[side == 0 ? TK_OB_H0 : TK_OB_H1];
#define CASE(SV)                                                                                                    \
  case SV:                                                                                                          \
    ob_reduce_hsplit_kernel<SV><<<counted(grid), NT, 0, strm>>>(st, partial, ncta, nb, H, ldh, row0, col0, Hc,      \
                                                                add ? 1 : 0, ticket, o.vexp, o.eh, (__half*)o.HB,   \
                                                                o.mx);                                              \
    break;
  switch (s) { SYLV_OB_S_CASES(CASE) }
#undef CASE
}

}  // namespace sylv
