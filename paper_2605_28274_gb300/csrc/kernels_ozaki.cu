// Float64 products of the small Sylvester operator on the tensor cores (Ozaki scheme I).
//
// The operator Q^ = [H P^, 0] + [P^ G^T; 0] of Algorithms 4.1/4.2 (eq. 3.7) is a dense
// contraction of order r (block upper Hessenberg H, G).  GB300 runs float64 FMAs at 1/64 of
// its FP32 rate, so the float64 kernel is bound by the FP64 pipe.  Here both factors are
// split exactly into BF16 integer digits and multiplied on the tcgen05 tensor cores:
//
//   x = 2^e * sum_{p=1..8} d_p 2^{-7p}   (e: exponent of the row's largest |x|; d_1 in
//                                         [-128, 128], d_p in [-64, 64]: exact in BF16)
//   (A B)_{ab} = 2^{e_a + f_b} sum_{p+q <= 9} 2^{-7(p+q)} (D^A_p D^B_q)_{ab}
//
// (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix multiplication by using
// fast routines of matrix multiplication and its applications", Numer. Algorithms 59, 2012;
// its tensor-core form: Mukunoki, Ozaki, Ogita, Imamura, ICCS 2020.)  Each digit product is
// an integer; the products of one level l = p + q over 128 values of k are below 2^23 in
// magnitude, so the FP32 accumulation in tensor memory is exact.  After every 128 values of
// k the eight level sums are added, as integers, into two int64 fixed-point accumulators
// (levels 2..5 in units of 2^-35, levels 6..9 in units of 2^-63; neither can overflow for
// k <= 2^13): the whole sum is exact, and the only rounding is the epilogue's conversion to
// float64.  The result differs from the exact product only by the digits dropped with the
// pairs p + q > 9, below 2^-56 of (max |row of A|)(max |column of B|) per term.
//
// Digits are stored in the canonical no-swizzle K-major layout of the tcgen05 shared-memory
// matrix descriptor (8-row x 16-byte core matrices), one 128 x 32 (A) or 64 x 32 (B) block
// per (digit, row tile, k stage), so plain 1-D bulk copies (cp.async.bulk) load each block.
// A CTA owns a 128 x 64 output tile and a range of its fold periods (exact k splits fill the
// GPU at small orders); two stage buffers let the copies of the next 32 values of k run during
// the MMAs of the current ones.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace sylv {

namespace {

constexpr int OZ_P = 8;               // digits per operand
constexpr int OZ_L = OZ_P + 1;        // pairs with p + q <= OZ_L are kept
constexpr int OZ_NLEV = OZ_L - 1;     // levels 2..OZ_L
constexpr int OZ_TM = 128;            // output rows per CTA (MMA M)
constexpr int OZ_TN = 64;             // output columns per CTA (MMA N)
constexpr int OZ_KC = 32;             // k per stage (one bulk copy per digit plane and operand)
constexpr int OZ_FOLD = 4;            // stages per fold (128 values of k)
constexpr int OZ_ABLK = OZ_TM * OZ_KC;  // BF16 elements of one A digit block (8 KB)
constexpr int OZ_BBLK = OZ_TN * OZ_KC;  // BF16 elements of one B digit block (4 KB)
constexpr int OZ_THREADS = 256;     // warps w and w + 4 share TMEM lanes 32 (w % 4) ..; each takes half the columns
constexpr int OZ_CPT = OZ_TN / 2;    // output columns per thread
constexpr int OZ_TMEM_COLS = OZ_NLEV * OZ_TN;  // one FP32 accumulator tile per level
static_assert(OZ_TMEM_COLS == 512, "tensor memory holds 512 columns");
constexpr int OZ_EXP_BAD = 1 << 20;   // exponent sentinel: the row holds a non-finite value
constexpr int OZ_OMEGA_CTAS = 1024;  // grid of the omega reduction (its partials live in the scratch)
constexpr int OZ_WAIT_ITERS = 1 << 20;
constexpr size_t OZ_STAGE = (size_t)OZ_P * (OZ_ABLK + OZ_BBLK) * 2;  // 96 KB
constexpr size_t OZ_SMEM = 2 * OZ_STAGE + 2048;  // two stages + 1 KB alignment, barriers
constexpr int OZ_MAX_SPLIT_CTAS = 4 * 152;  // k-split partials are kept for at most this many CTAs

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor, no swizzle: start address, leading-dimension
// byte offset (between core matrices adjacent in k), stride byte offset (between 8-row groups).
__device__ __forceinline__ uint64_t oz_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture family
  return d;
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, M x N.
constexpr uint32_t oz_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Offset (in BF16 elements) of element (i, k) inside one T x 64 digit block.
__device__ __forceinline__ int oz_in_block(int i, int k) {
  return (((i >> 3) * (OZ_KC / 8) + (k >> 3)) << 6) + ((i & 7) << 3) + (k & 7);
}

// mx[i] = max_k |x(i, k)| as IEEE bits (non-negative doubles order like their bit patterns);
// x(i, k) = X[i * si + k * sk], i < R, k < K.  A CTA covers 32 rows x 64 values of k (8 per
// thread) and combines into mx (zeroed beforehand) with atomicMax: the result does not depend
// on the order.
__device__ __forceinline__ void oz_max_body(const double* __restrict__ X, int64_t si, int64_t sk, int R, int K,
                                            unsigned long long* __restrict__ mx) {
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int k0 = blockIdx.y * 64 + (threadIdx.x >> 5) * 8;
  if (i >= R) return;
  unsigned long long m = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int k = k0 + j;
    if (k < K)
      m = max(m, (unsigned long long)__double_as_longlong(X[(int64_t)i * si + (int64_t)k * sk]) & 0x7FFFFFFFFFFFFFFFull);
  }
  if (m) atomicMax(mx + i, m);
}

// e = 1 + floor(log2 m) (0 for a zero or subnormal-only row, OZ_EXP_BAD for a non-finite one)
__device__ __forceinline__ int oz_exponent(unsigned long long m) {
  if (m >= 0x7FF0000000000000ull) return OZ_EXP_BAD;
  if (m < 0x0010000000000000ull) return 0;
  return (int)(m >> 52) - 1023 + 1;
}

// Digits of x(i, k) for one row i and 8 consecutive k: thread per (i, k group).  Writes the
// 8 digit planes, each as one 16-byte core-matrix row.  Layout of a plane: blocks
// [row tile][k chunk] of T x 64, T = rows per tile.
__device__ __forceinline__ void oz_split_body(const double* __restrict__ X, int64_t si, int64_t sk, int R, int K,
                                              int Rp, int Kp, int T, const unsigned long long* __restrict__ mx,
                                              int* __restrict__ ex, __nv_bfloat16* __restrict__ dig, int64_t plane) {
  const int kg_n = Kp / 8;
  const int64_t t = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (t >= (int64_t)Rp * kg_n) return;
  const int i = (int)(t % Rp), kg = (int)(t / Rp);  // consecutive threads: consecutive rows
  const int e = i < R ? oz_exponent(mx[i]) : 0;
  if (kg == 0) ex[i] = e;
  long long Nv[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int k = kg * 8 + j;
    double x = 0.0;
    if (i < R && k < K && e != OZ_EXP_BAD) x = X[(int64_t)i * si + (int64_t)k * sk];
    // N = x 2^{56-e} rounded to the nearest integer (ties to even); |x| < 2^e, so |N| <= 2^56.
    // Integer operations on the IEEE bits only: the FP64 pipe of this GPU is narrow.
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    long long N = 0;
    if (ex != 0x7FF && (bits & 0x7FFFFFFFFFFFFFFFull) != 0) {
      // x = mant 2^{ex - 1075} (a subnormal x: no implicit bit, exponent field 1)
      const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (ex != 0 ? (1ull << 52) : 0ull);
      const int sh = (ex != 0 ? ex : 1) - 1075 + 56 - e;  // N = mant 2^sh, sh <= 3
      unsigned long long u;
      if (sh >= 0) {
        u = mant << sh;
      } else if (sh < -54) {
        u = 0;
      } else {
        const int rs = -sh;
        const unsigned long long q = mant >> rs, rem = mant & ((1ull << rs) - 1), half = 1ull << (rs - 1);
        u = q + ((rem > half || (rem == half && (q & 1))) ? 1ull : 0ull);
      }
      N = (bits >> 63) ? -(long long)u : (long long)u;
    }
    Nv[j] = N;
  }
  const int nkc = Kp / OZ_KC;
  const int64_t blk = ((int64_t)(i / T) * nkc + (kg * 8) / OZ_KC) * ((int64_t)T * OZ_KC);
  const int inb = oz_in_block(i % T, (kg * 8) % OZ_KC);
#pragma unroll
  for (int p = 1; p <= OZ_P; ++p) {
    const int sh = 7 * (OZ_P - p);
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      long long d;
      if (sh > 0) {
        d = (Nv[j] + (1ll << (sh - 1))) >> sh;  // nearest multiple of 2^sh (ties up)
        Nv[j] -= d << sh;
      } else {
        d = Nv[j];
      }
      v[j] = __float2bfloat16_rn(__int2float_rn((int)d));  // |d| <= 128: exact
    }
    *reinterpret_cast<uint4*>(dig + (int64_t)(p - 1) * plane + blk + inb) = *reinterpret_cast<const uint4*>(v);
  }
}

// The four operands of one small-operator call (pass 1: H, Z; pass 2: Z, G^T), so that their
// column maxima and their digits take one launch each instead of four.
struct OzOp {
  const double* X;  // x(i, k) = X[i si + k sk], i < R, k < K
  int64_t si, sk;
  int R, Rp, T;     // rows, rows padded to the tile, rows per tile
  unsigned long long* mx;
  int* ex;
  __nv_bfloat16* dig;
  int64_t plane;
};
struct OzOps {
  OzOp op[4];
  int K, Kp;
};

// Column maxima of the four operands: blockIdx.z selects the operand; CTAs beyond an
// operand's extent find no rows or no k and return without writing.
__global__ void __launch_bounds__(NT) oz_max4_kernel(const DevState* st, OzOps ops) {
  if (stopped(st)) return;
  const OzOp& o = ops.op[blockIdx.z];
  oz_max_body(o.X, o.si, o.sk, o.R, ops.K, o.mx);
}

// Digits of the four operands: blockIdx.y selects the operand (threads beyond its padded
// extent return).
__global__ void __launch_bounds__(NT) oz_split4_kernel(const DevState* st, OzOps ops) {
  if (stopped(st)) return;
  const OzOp& o = ops.op[blockIdx.y];
  oz_split_body(o.X, o.si, o.sk, o.R, ops.K, o.Rp, ops.Kp, o.T, o.mx, o.ex, o.dig, o.plane);
}

__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t phase) {
  for (int it = 0; it < OZ_WAIT_ITERS; ++it) {
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

// v: an FP32 level sum, an exact integer below 2^22 in magnitude.  Its integer value comes
// from the bits of v + 1.5 * 2^23 (exact for |v| < 2^22).
__device__ __forceinline__ int oz_int(float v) {
  return __float_as_int(__fadd_rn(v, 12582912.0f)) - 0x4B400000;
}

// Out[a + b*ldo] (= or +=) 2^{e_a + f_b} sum_k A(a, k) B(b, k) over the tile's k range.
// A digits: planes of Mp x Kp (tiles of 128 rows), B digits: Np x Kp (tiles of 64 rows).
// hess: 0 all k stages; 1 start at the block-Hessenberg bound of the tile's first row
// (A = H); 2 the same for the tile's first column (B = G^T).  Valid outputs a < Mv, b < Nv.
// blockIdx.z splits the tile's fold periods into gridDim.z ranges; with more than one, each CTA
// writes its exact int64 fixed-point sums to part (oz_reduce_kernel adds them and writes Out).
// Stages of 32 values of k are double-buffered: the bulk copies of the next stage run during
// this stage's MMAs.  One thread issues the 72 MMAs of a stage from descriptors computed once
// and advanced by constant offsets (issuing, not the tensor pipe, bounds MMAs this narrow).
// A wait that gives up sets the solve status to ST_WAIT_TIMEOUT.
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_gemm_kernel(
    DevState* st, const __nv_bfloat16* __restrict__ Ad, int64_t planeA, const __nv_bfloat16* __restrict__ Bd,
    int64_t planeB, int nkc, const int* __restrict__ ea, const int* __restrict__ fb, int hess, int s, double* Out,
    int64_t ldo, int Mv, int Nv, int add, long long* __restrict__ part) {
  if (stopped(st)) return;
  extern __shared__ __align__(1024) unsigned char oz_smem[];
  unsigned char* base = (unsigned char*)(((uintptr_t)oz_smem + 1023) & ~(uintptr_t)1023);
  // stage b: A planes at base + b * OZ_STAGE, B planes after them
  uint64_t* bars = (uint64_t*)(base + 2 * OZ_STAGE);  // [0], [1] loads of stage 0 / 1, [2] MMAs
  uint32_t* tmem_slot = (uint32_t*)(bars + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, nt = blockIdx.y;
  const int a0 = mt * OZ_TM, b0 = nt * OZ_TN;

  int kc0 = 0;
  if (hess == 1) kc0 = max(0, (a0 / s - 1) * s) / OZ_KC;
  if (hess == 2) kc0 = max(0, (b0 / s - 1) * s) / OZ_KC;
  // fold periods start at multiples of OZ_FOLD stages, so each covers at most OZ_FOLD stages
  kc0 -= kc0 % OZ_FOLD;
  // this CTA's fold periods
  const int periods = (nkc - kc0 + OZ_FOLD - 1) / OZ_FOLD;
  const int per_split = (periods + (int)gridDim.z - 1) / (int)gridDim.z;
  const int kb = kc0 + (int)blockIdx.z * per_split * OZ_FOLD;
  const int ke = min(nkc, kb + per_split * OZ_FOLD);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(OZ_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  const uint32_t bar_ld0 = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[2]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_ld0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_ld0 + 8));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_mma));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  const int quarter = warp & 3, col0 = (warp >> 2) * OZ_CPT;  // TMEM lanes 32 quarter .., columns col0 ..
  long long w1[OZ_CPT], w2[OZ_CPT];  // levels 2..5 (unit 2^-35) and 6..9 (unit 2^-63)
#pragma unroll
  for (int j = 0; j < OZ_CPT; ++j) w1[j] = w2[j] = 0;

  const uint32_t id = oz_idesc(OZ_TM, OZ_TN);
  const uint32_t lbo = 128, sbo = (OZ_KC / 8) * 128;
  constexpr uint32_t abytes = OZ_ABLK * 2, bbytes = OZ_BBLK * 2;
  // stage kc's copies into buffer (kc - kb) & 1 (thread 0)
  auto load = [&](int kc) {
    const int b = (kc - kb) & 1;
    unsigned char* sA = base + (size_t)b * OZ_STAGE;
    unsigned char* sB = sA + (size_t)OZ_P * abytes;
    const uint32_t bar = bar_ld0 + 8 * b;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(OZ_P * (abytes + bbytes))
                 : "memory");
#pragma unroll 1
    for (int p = 0; p < OZ_P; ++p) {
      const __nv_bfloat16* ga = Ad + (int64_t)p * planeA + ((int64_t)mt * nkc + kc) * OZ_ABLK;
      const __nv_bfloat16* gb = Bd + (int64_t)p * planeB + ((int64_t)nt * nkc + kc) * OZ_BBLK;
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(sA + (size_t)p * abytes)),
                   "l"(ga), "r"(abytes), "r"(bar)
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(sB + (size_t)p * bbytes)),
                   "l"(gb), "r"(bbytes), "r"(bar)
                   : "memory");
    }
  };
  if (tid == 0 && kb < ke) load(kb);
  bool ok = true;
  uint32_t stuck_bar = 0, stuck_phase = 0;  // barrier whose wait gave up (0: none)
  int next_stage = -1;                      // thread 0: the stage whose copies it issued ahead
  for (int kc = kb; kc < ke && ok; ++kc) {
    const int i = kc - kb, b = i & 1;
    const bool first_of_fold = (i % OZ_FOLD) == 0;
    const bool last_of_fold = (i % OZ_FOLD) == OZ_FOLD - 1 || kc == ke - 1;
    // the other buffer is free: the MMAs of stage kc - 1 completed in the previous iteration
    if (tid == 0 && kc + 1 < ke) {
      load(kc + 1);
      next_stage = kc + 1;
    }
    const uint32_t ph_ld = (uint32_t)(i >> 1) & 1u;
    ok = __syncthreads_and(oz_wait(bar_ld0 + 8 * b, ph_ld));
    if (!ok) {
      stuck_bar = bar_ld0 + 8 * b;
      stuck_phase = ph_ld;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      // level l = p + q accumulates in TMEM columns (l - 2) * 64 ..; its first MMA of a fold
      // period overwrites (p = 1 comes first for every level)
      const uint32_t sA = smem_u32(base + (size_t)b * OZ_STAGE);
      const uint64_t dA = oz_sdesc(sA, lbo, sbo), dB = oz_sdesc(sA + OZ_P * abytes, lbo, sbo);
#pragma unroll
      for (int p = 1; p <= OZ_P; ++p)
#pragma unroll
        for (int q = 1; q <= OZ_L - p; ++q)
#pragma unroll
          for (int ks = 0; ks < OZ_KC / 16; ++ks) {
            const uint32_t acc = (first_of_fold && p == 1 && ks == 0) ? 0u : 1u;
            asm volatile(
                "{\n .reg .pred pa;\n setp.ne.b32 pa, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}\n" ::"r"(
                    tmem + (uint32_t)((p + q - 2) * OZ_TN)),
                "l"(dA + (uint64_t)(((p - 1) * abytes + ks * 256) >> 4)),
                "l"(dB + (uint64_t)(((q - 1) * bbytes + ks * 256) >> 4)), "r"(id), "r"(acc)
                : "memory");
          }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_mma)
                   : "memory");
    }
    const uint32_t ph_mma = (uint32_t)i & 1u;
    ok = __syncthreads_and(oz_wait(bar_mma, ph_mma));
    if (!ok) {
      stuck_bar = bar_mma;
      stuck_phase = ph_mma;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (last_of_fold) {
#pragma unroll
      for (int l = 2; l <= OZ_L; ++l) {
        const int sh = l <= 5 ? 7 * (5 - l) : 7 * (9 - l);
#pragma unroll
        for (int c = 0; c < OZ_CPT; c += 16) {
          uint32_t r[16];
          const uint32_t addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((l - 2) * OZ_TN + col0 + c);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                "=r"(r[15])
              : "r"(addr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const long long t = (long long)((unsigned long long)(long long)oz_int(__uint_as_float(r[j])) << sh);
            if (l <= 5)
              w1[c + j] += t;
            else
              w2[c + j] += t;
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // tensor memory and this stage's buffer are free for the next stages
  }

  if (ok) {
    const int arow = quarter * 32 + lane, a = a0 + arow;
    if (gridDim.z > 1) {
      // exact partial sums of this k range: [split][tile][column][row] x (w1, w2), rows fastest
      // (the lanes of a warp hold consecutive rows: coalesced here and in oz_reduce_kernel)
      const int64_t tile = (int64_t)blockIdx.z * gridDim.x * gridDim.y + (int64_t)mt * gridDim.y + nt;
#pragma unroll
      for (int j = 0; j < OZ_CPT; ++j) {
        longlong2* o = (longlong2*)part + (tile * OZ_TN + col0 + j) * OZ_TM + arow;
        *o = make_longlong2(w1[j], w2[j]);
      }
    } else if (a < Mv) {
      const int e = ea[a];
#pragma unroll
      for (int j = 0; j < OZ_CPT; ++j) {
        const int b = b0 + col0 + j;
        if (b < Nv) {
          const int f = fb[b];
          const int x = e + f;  // 2^x as a float64 (x outside the normal range: 0 or inf)
          const double sc = x < -1022 ? 0.0 : (x > 1023 ? __longlong_as_double(0x7FF0000000000000ll)
                                                        : __longlong_as_double((long long)(x + 1023) << 52));
          double v = fma((double)w1[j], 0x1p-35, (double)w2[j] * 0x1p-63) * sc;
          if (e == OZ_EXP_BAD || f == OZ_EXP_BAD) v = __longlong_as_double(0x7FF8000000000000ll);
          double* o = Out + a + (int64_t)b * ldo;
          *o = add ? (*o + v) : v;
        }
      }
    }
  } else {
    if (tid == 0) {
      st->breakdown_where = 200;
      atomicExch(&st->status, (int)ST_WAIT_TIMEOUT);
    }
    // copies or MMAs that timed out may still be in flight: a second bounded wait before the
    // shared memory and the tensor memory are given up, and one for the copies of the stage
    // issued ahead
    oz_wait(stuck_bar, stuck_phase);
    if (tid == 0 && next_stage >= 0) {
      const int j = next_stage - kb;
      oz_wait(bar_ld0 + 8 * (j & 1), (uint32_t)(j >> 1) & 1u);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS));
}

// Out (= or +=) the sum over the k splits of the exact partial sums, scaled by 2^{e_a + f_b}.
__global__ void __launch_bounds__(NT) oz_reduce_kernel(DevState* st, const long long* __restrict__ part, int splits,
                                                       int tm, int tn, const int* __restrict__ ea,
                                                       const int* __restrict__ fb, double* Out, int64_t ldo, int Mv,
                                                       int Nv, int add) {
  if (stopped(st)) return;
  const int64_t t = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (t >= (int64_t)Mv * Nv) return;
  const int a = (int)(t % Mv), b = (int)(t / Mv);  // consecutive threads: consecutive rows (Out is column-major)
  const int64_t tile = (int64_t)(a / OZ_TM) * tn + b / OZ_TN;
  const int64_t idx = (tile * OZ_TN + b % OZ_TN) * OZ_TM + a % OZ_TM;
  const int64_t stride = (int64_t)tm * tn * OZ_TM * OZ_TN;
  long long w1 = 0, w2 = 0;
  for (int z = 0; z < splits; ++z) {
    const longlong2 v = ((const longlong2*)part)[z * stride + idx];
    w1 += v.x;
    w2 += v.y;
  }
  const int e = ea[a], f = fb[b];
  const int x = e + f;
  const double sc = x < -1022 ? 0.0 : (x > 1023 ? __longlong_as_double(0x7FF0000000000000ll)
                                                : __longlong_as_double((long long)(x + 1023) << 52));
  double v = fma((double)w1, 0x1p-35, (double)w2 * 0x1p-63) * sc;
  if (e == OZ_EXP_BAD || f == OZ_EXP_BAD) v = __longlong_as_double(0x7FF8000000000000ll);
  double* o = Out + a + (int64_t)b * ldo;
  *o = add ? (*o + v) : v;
}

// <Out(1:r,1:r), Z> and <Out, Out> over the rp x rp extent; the last CTA sets omega.
__global__ void __launch_bounds__(NT) oz_omega_kernel(DevState* st, int r, int rp, const double* __restrict__ Out,
                                                      const double* __restrict__ Z, int64_t lds,
                                                      double* __restrict__ partials) {
  if (stopped(st)) return;
  __shared__ double sh[32];
  __shared__ int last_sh;
  double ts = 0.0, tt = 0.0;
  const int64_t E = (int64_t)rp * rp;
  for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < E; e += (int64_t)gridDim.x * NT) {
    const int a = (int)(e % rp), b = (int)(e / rp);
    const double v = Out[a + (int64_t)b * lds];
    tt += v * v;
    if (a < r && b < r) ts += v * Z[a + (int64_t)b * lds];
  }
  ts = block_sum(ts, sh);
  tt = block_sum(tt, sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = ts;
    partials[2 * blockIdx.x + 1] = tt;
  }
  if (last_cta(&st->tickets[TK_BI_T], &last_sh)) {
    const double s1 = cta_sum(partials, (int)gridDim.x, 2, 0, sh), s2 = cta_sum(partials, (int)gridDim.x, 2, 1, sh);
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

int oz_pad(int x, int t) { return (x + t - 1) / t * t; }

}  // namespace

size_t ozaki_scratch_bytes(int rmax) {
  const int Mp = oz_pad(rmax, OZ_TM), Kp = oz_pad(rmax, OZ_KC * OZ_FOLD);
  // two passes x two digit sets (A and B operand) of Mp x Kp BF16 x 8 planes, their exponents,
  // column maxima, omega partials, k-split partial sums (two int64 per output of at most
  // OZ_MAX_SPLIT_CTAS tiles)
  return (size_t)4 * OZ_P * Mp * Kp * 2 + (size_t)4 * Mp * sizeof(int) + (size_t)4 * Mp * sizeof(unsigned long long) +
         (size_t)2 * OZ_OMEGA_CTAS * sizeof(double) + (size_t)OZ_MAX_SPLIT_CTAS * OZ_TM * OZ_TN * 2 * sizeof(long long) +
         1024;
}

bool ozaki_setup() {
  return cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM) ==
         cudaSuccess;
}

// Out(rp x rp, ld lds) = [H Z, 0] + [Z G^T; 0]: two tensor-core passes, each after splitting its
// two operands.  scratch: ozaki_scratch_bytes(rp) bytes.  Returns the number of kernels launched.
int launch_sylv_gemm_ozaki(cudaStream_t strm, DevState* st, int r, int s, const double* H, const double* G,
                           int64_t ldh, const double* Z, double* Out, int64_t lds, bool omega, void* scratch) {
  const int rp = r + s;
  const int Mp = oz_pad(rp, OZ_TM);           // A rows (output rows)
  const int Np = oz_pad(rp, OZ_TN);           // B rows (output columns)
  const int Kp = oz_pad(r, OZ_KC * OZ_FOLD);  // contraction length
  const int nkc = Kp / OZ_KC;
  const int64_t planeA = (int64_t)Mp * Kp, planeB = (int64_t)Np * Kp;
  // digits of both passes' operands (pass 1: A = H, B = Z; pass 2: A = Z, B = G^T), split up front
  __nv_bfloat16* Ad1 = (__nv_bfloat16*)scratch;
  __nv_bfloat16* Bd1 = Ad1 + (size_t)OZ_P * planeA;
  __nv_bfloat16* Ad2 = Bd1 + (size_t)OZ_P * planeB;
  __nv_bfloat16* Bd2 = Ad2 + (size_t)OZ_P * planeA;
  int* ea1 = (int*)(Bd2 + (size_t)OZ_P * planeB);
  int* fb1 = ea1 + Mp;
  int* ea2 = fb1 + Mp;
  int* fb2 = ea2 + Mp;
  unsigned long long* mx = (unsigned long long*)(((uintptr_t)(fb2 + Mp) + 15) & ~(uintptr_t)15);  // 4 x Mp
  double* partials = (double*)(mx + 4 * (size_t)Mp);
  long long* kpart = (long long*)(((uintptr_t)(partials + 2 * OZ_OMEGA_CTAS) + 255) & ~(uintptr_t)255);
  // k splits: the tiles alone leave SMs idle at most orders (28 tiles at r = 448); split each
  // tile's fold periods so that the CTAs fill the GPU in whole waves, within the partial buffer
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  const int tm = Mp / OZ_TM, tn = Np / OZ_TN, tiles = tm * tn;
  const int periods = Kp / (OZ_KC * OZ_FOLD);
  int ks = 1;
  double best = 1e30;
  for (int z = 1; z <= 8 && z <= periods && z * tiles <= OZ_MAX_SPLIT_CTAS; ++z) {
    const double waves = (double)((tiles * z + sms - 1) / sms) / z + 0.02 * z;  // per unit of tile work
    if (waves < best) {
      best = waves;
      ks = z;
    }
  }
  const dim3 grid(tm, tn, ks);
  const unsigned gr = (unsigned)(((int64_t)rp * rp + NT - 1) / NT);
  const dim3 gmA((unsigned)((rp + 31) / 32), (unsigned)((r + 63) / 64));
  const unsigned gsA = (unsigned)(((int64_t)Mp * (Kp / 8) + NT - 1) / NT);
  cudaMemsetAsync(mx, 0, (size_t)4 * Mp * sizeof(unsigned long long), strm);
  // pass 1: Out = H Z  (A(a, c) = H[a + c ldh], B(b, c) = Z[c + b lds]), all rp x rp outputs;
  // pass 2: Out += Z G^T  (A(a, c) = Z[a + c lds], B(b, c) = G[b + c ldh]), rows a < r
  OzOps ops{};
  ops.K = r;
  ops.Kp = Kp;
  ops.op[0] = {H, 1, ldh, rp, Mp, OZ_TM, mx, ea1, Ad1, planeA};
  ops.op[1] = {Z, lds, 1, r, Np, OZ_TN, mx + Mp, fb1, Bd1, planeB};
  ops.op[2] = {Z, 1, lds, r, Mp, OZ_TM, mx + 2 * (size_t)Mp, ea2, Ad2, planeA};
  ops.op[3] = {G, 1, ldh, rp, Np, OZ_TN, mx + 3 * (size_t)Mp, fb2, Bd2, planeB};
  oz_max4_kernel<<<counted(dim3(gmA.x, gmA.y, 4)), NT, 0, strm>>>(st, ops);
  oz_split4_kernel<<<counted(dim3(gsA, 4)), NT, 0, strm>>>(st, ops);
  oz_gemm_kernel<<<counted(grid), OZ_THREADS, OZ_SMEM, strm>>>(st, Ad1, planeA, Bd1, planeB, nkc, ea1, fb1, 1, s, Out,
                                                               lds, rp, rp, 0, kpart);
  if (ks > 1) oz_reduce_kernel<<<counted(gr), NT, 0, strm>>>(st, kpart, ks, tm, tn, ea1, fb1, Out, lds, rp, rp, 0);
  oz_gemm_kernel<<<counted(grid), OZ_THREADS, OZ_SMEM, strm>>>(st, Ad2, planeA, Bd2, planeB, nkc, ea2, fb2, 2, s, Out,
                                                               lds, r, rp, 1, kpart);
  if (ks > 1) oz_reduce_kernel<<<counted(gr), NT, 0, strm>>>(st, kpart, ks, tm, tn, ea2, fb2, Out, lds, r, rp, 1);
  int launched = ks > 1 ? 6 : 4;
  if (omega) {
    const int64_t E = (int64_t)rp * rp;
    const unsigned g = (unsigned)std::min<int64_t>((E + NT - 1) / NT, OZ_OMEGA_CTAS);
    oz_omega_kernel<<<counted(g), NT, 0, strm>>>(st, r, rp, Out, Z, lds, partials);
    launched += 1;
  }
  return launched;
}

}  // namespace sylv
