// C ABI of libsylv: handle management, device memory, and the host drivers of
// factorized CG (Algorithm 4.1) and factorized BiCGSTAB (Algorithm 4.2).
//
// The host only enqueues kernels: every scalar of the recurrences stays on the
// device (DevState) and every kernel is a no-op once the device status says the
// solve stopped.  The host copies the status back once every `poll_every`
// iterations, one chunk behind the enqueue point, so the GPU never idles
// waiting for the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/sylv.h"
#include "common.cuh"
#include "kernels.h"

using sylv::DevState;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CU(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      if (e_ == cudaErrorMemoryAllocation) {                                                  \
        cudaGetLastError();                                                                   \
        return fail(SYLV_ENOMEM, std::string(#call) + ": " + cudaGetErrorString(e_));         \
      }                                                                                       \
      return fail(SYLV_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
    }                                                                                         \
  } while (0)

#define TRY(expr)            \
  do {                       \
    int rc_ = (expr);        \
    if (rc_ != SYLV_OK) return rc_; \
  } while (0)

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Side {
  int64_t n = 0, nnz = 0;
  int32_t* rp = nullptr;
  int32_t* ci = nullptr;
  double* vald = nullptr;
  float* valf = nullptr;
  double* C = nullptr;  // n x s column-major, float64
  void* V = nullptr;    // maxb blocks, block-row-major, factor precision
  double* H = nullptr;  // ldh x ldh column-major
  double* RQR = nullptr;
  double* R1 = nullptr;
  double* Rinv = nullptr;
  void* RinvT = nullptr;
  sylv::ObSide ob;  // float64 Arnoldi basis as tensor-core digit planes (G == nullptr: not used)
};

enum Method { M_NONE = 0, M_CG = 1, M_BICG = 2, M_CGS = 3, M_CR = 4, M_GPBICG = 5 };  // CR: Lanczos, others Arnoldi
inline bool arnoldi_method(int m) { return m == M_BICG || m == M_CGS || m == M_GPBICG; }
inline bool lanczos_method(int m) { return m == M_CG || m == M_CR; }

// Kernel classes timed by the optional profiler.
enum KClass {
  KC_SPMM = 0, KC_GRAM, KC_REDUCE, KC_UPDATE, KC_CHOL, KC_SCALE, KC_SETUP,
  KC_SMALL_GEMM, KC_SMALL_OP, KC_SMALL_ELEM, KC_RESID, KC_RESID_TSG, KC_RESID_TSU, KC_RESID_SMALL,
  KC_RESID_SPMM, KC_RESID_QR, KC_RESID_MISC, KC_BSPLIT, KC_NUM
};
const char* const kKcNames[KC_NUM] = {"spmm",         "gram",  "reduce_h",   "update",           "cholqr_chol",
                                      "cholqr_scale", "setup", "small_gemm", "small_op_tridiag", "small_elementwise",
                                      "true_residual", "resid_tsg", "resid_tsu", "resid_small", "resid_spmm",
                                      "resid_qr", "resid_misc", "basis_split"};

struct Prof {
  struct Rec {
    int cls, k;
    cudaEvent_t a, b;
    double bytes, flops;
  };
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<Rec> recs;
  int64_t launches[KC_NUM] = {};
  double ms[KC_NUM] = {}, bytes[KC_NUM] = {}, flops[KC_NUM] = {};
  int cur_k = -1;
  bool valid = false;
  size_t flushed = 0;  // records already summed
};

}  // namespace

namespace sylv {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace sylv

struct sylv_handle {
  sylv_options opt{};
  int64_t s = 0;
  bool lyap = false, mixed = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Side side[2];
  std::vector<void*> fixed_allocs, solve_allocs;
  // per-solve capacity
  int maxb = 0, cap_method = M_NONE;
  int64_t lds = 0;
  double *Xh = nullptr, *Rh = nullptr, *Ph = nullptr, *Qh = nullptr, *Sh = nullptr, *Th = nullptr, *Rt = nullptr;
  double* Uh = nullptr;  // CGS, GPBiCG
  double *gW = nullptr, *gZ = nullptr, *gTp = nullptr, *gY = nullptr, *gPart = nullptr;  // GPBiCG only
  DevState* st = nullptr;
  DevState* st_host = nullptr;  // pinned, 2 slots
  double* hist = nullptr;
  int hist_cap = 0;
  double* spart = nullptr;   // self-Gram partials
  double* spart2 = nullptr;  // the same, written by a fused CholQR pass that reads spart
  double* psmall = nullptr;
  // mixed mode: hi/lo float pairs of H, G and of the small operand (8 bytes per entry)
  double *Hs = nullptr, *Gs = nullptr, *Zs = nullptr;
  int split_cols = 0;  // columns of H, G split so far in this solve
  void* oz_scratch = nullptr;  // digit planes of the tensor-core small products
  bool ob_unavailable = false;  // the basis digit planes did not fit: CUDA-core basis kernels
  // sylv_compress: rank-q factors (column-major, device) that sylv_get_factors returns until the
  // next solve; comp_q < 0: not compressed
  double *comp_V = nullptr, *comp_W = nullptr;
  std::vector<double> comp_s;
  int64_t comp_q = -1;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  Prof prof;
  cudaStream_t prof_stream = nullptr;  // stream the profiler records on (null: h->stream)
  int64_t launches = 0;  // kernels enqueued by the current solve
  // the two block Krylov bases run on their own streams, ahead of the small side
  cudaStream_t sbas[2] = {nullptr, nullptr};
  double *gpart_s[2] = {nullptr, nullptr}, *spart_s[2] = {nullptr, nullptr}, *Hc_s[2] = {nullptr, nullptr};
  double* spart2_s[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_bas[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}}, ev_small[8] = {};
  // last solve
  int method = M_NONE;
  int iters = 0;
  int status = -1;
  int64_t width = 0;
  int nblocks = 0;
  // float64 true residual (randomised sketch) and mixed-precision refinement
  Side opAt, opB;                  // CSR of A^T and of B (float64) for R^T Q and R Omega
  double* C1rm = nullptr;          // C1, C2 row-major float64 (n x s, m x s)
  double* C2rm = nullptr;
  double* Om = nullptr;            // two m x 8 Gaussian probe blocks (row-major)
  double cnorm = -1.0;             // ||C1 C2^T||_F
  DevState* st_sk = nullptr;       // status word of the sketch's CholQR
  double* sk_host = nullptr;       // pinned: 3 sums + the sketch's DevState
  std::vector<std::pair<void*, size_t>> sk;  // sketch scratch buffers (pointer, bytes)
  std::vector<sylv_handle*> subs;  // correction solves of the last mixed solve
  bool is_sub = false;
  // the last solve's bases as digit planes for the certificate's products (float32 bases, or
  // float64 ones kept on the CUDA cores); built at the first certificate after a solve
  void* cert_mem = nullptr;
  size_t cert_bytes = 0;
  sylv::ObSide cert_ob[2];
  bool cert_valid = false, cert_failed = false;
  int64_t cert_R = 0;            // basis columns the planes hold
  const void* cert_V = nullptr;  // side 0's basis they were split from
  // batched Lyapunov CG: one internal handle per instance
  std::vector<sylv_handle*> batch;
  sylv::BatchInst* d_insts = nullptr;
  int2* d_items = nullptr;
  double *b_gpart = nullptr, *b_spart = nullptr;
  int* d_running = nullptr;
  int* h_running = nullptr;  // pinned, 2 slots
  size_t items_cap = 0;
  int tuned_chunk = 0, tuned_grid = 0;
  std::vector<cudaStream_t> pool;  // streams for the per-instance true-residual sketches
  double tune_ms = 0.0;
  cudaGraphExec_t graph = nullptr;
  double true_rel = -1.0;    // estimate of the float64 true relative residual
  double true_bound = -1.0;  // its certified upper bound (probability >= 1 - kCertDelta)
  int refinements = 0;
  int64_t total_iters = 0, total_width = 0;
};

namespace {

int dev_alloc(sylv_handle* h, std::vector<void*>& list, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? SYLV_ENOMEM : SYLV_ECUDA,
                std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  list.push_back(*p);
  return SYLV_OK;
}

template <typename P>
int alloc_fixed(sylv_handle* h, P** p, size_t count) {
  return dev_alloc(h, h->fixed_allocs, (void**)p, count * sizeof(P));
}
template <typename P>
int alloc_solve(sylv_handle* h, P** p, size_t count) {
  return dev_alloc(h, h->solve_allocs, (void**)p, count * sizeof(P));
}

void free_compressed(sylv_handle* h) {
  if (h->comp_V) cudaFree(h->comp_V);
  if (h->comp_W) cudaFree(h->comp_W);
  h->comp_V = h->comp_W = nullptr;
  h->comp_s.clear();
  h->comp_q = -1;
}

void free_solve(sylv_handle* h) {
  for (void* p : h->solve_allocs) cudaFree(p);
  h->solve_allocs.clear();
  h->maxb = 0;
  h->cap_method = M_NONE;
  for (auto& sd : h->side) {
    sd.V = nullptr;
    sd.H = nullptr;
    sd.ob = sylv::ObSide{};
  }
  h->Hs = h->Gs = h->Zs = nullptr;
  h->Uh = nullptr;
  h->gW = h->gZ = h->gTp = h->gY = h->gPart = nullptr;
  h->oz_scratch = nullptr;
}

int check_csr(const sylv_csr* M, const char* name, int64_t expect_n) {
  if (M == nullptr) return fail(SYLV_EINVAL, std::string(name) + " is NULL");
  if (M->nrows <= 0 || M->ncols != M->nrows) return fail(SYLV_EINVAL, std::string(name) + " must be square and non-empty");
  if (expect_n >= 0 && M->nrows != expect_n) return fail(SYLV_EINVAL, std::string(name) + " has the wrong size");
  if (M->nrows > INT32_MAX - 1 || M->nnz < 0 || M->nnz > INT32_MAX)
    return fail(SYLV_EINVAL, std::string(name) + ": sizes exceed int32 indexing");
  if (!M->row_ptr || (M->nnz > 0 && (!M->col_idx || !M->val))) return fail(SYLV_EINVAL, std::string(name) + ": NULL arrays");
  if (M->row_ptr[0] != 0 || M->row_ptr[M->nrows] != M->nnz) return fail(SYLV_EINVAL, std::string(name) + ": bad row_ptr ends");
  for (int64_t i = 0; i < M->nrows; ++i)
    if (M->row_ptr[i + 1] < M->row_ptr[i]) return fail(SYLV_EINVAL, std::string(name) + ": row_ptr decreases");
  for (int64_t p = 0; p < M->nnz; ++p)
    if (M->col_idx[p] < 0 || M->col_idx[p] >= M->ncols) return fail(SYLV_EINVAL, std::string(name) + ": column index out of range");
  return SYLV_OK;
}

// Upload Op (A, or B^T built on the host by a counting sort) to the device.
int upload_operator(sylv_handle* h, Side& sd, const sylv_csr* M, bool transpose) {
  const int64_t n = M->nrows, nnz = M->nnz;
  std::vector<int32_t> rp(n + 1), ci(nnz);
  std::vector<double> val(nnz);
  if (!transpose) {
    std::copy(M->row_ptr, M->row_ptr + n + 1, rp.begin());
    std::copy(M->col_idx, M->col_idx + nnz, ci.begin());
    std::copy(M->val, M->val + nnz, val.begin());
  } else {
    std::vector<int64_t> cnt(n + 1, 0);
    for (int64_t p = 0; p < nnz; ++p) cnt[M->col_idx[p] + 1]++;
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    for (int64_t i = 0; i <= n; ++i) rp[i] = (int32_t)cnt[i];
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = M->row_ptr[i]; p < M->row_ptr[i + 1]; ++p) {
        const int64_t q = pos[M->col_idx[p]]++;
        ci[q] = (int32_t)i;
        val[q] = M->val[p];
      }
  }
  for (double v : val)
    if (!std::isfinite(v)) return fail(SYLV_ENONFINITE, "non-finite matrix entry");
  sd.n = n;
  sd.nnz = nnz;
  TRY(alloc_fixed(h, &sd.rp, n + 1));
  TRY(alloc_fixed(h, &sd.ci, std::max<int64_t>(nnz, 1)));
  TRY(alloc_fixed(h, &sd.vald, std::max<int64_t>(nnz, 1)));
  CU(cudaMemcpyAsync(sd.rp, rp.data(), (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
  if (nnz) {
    CU(cudaMemcpyAsync(sd.ci, ci.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(sd.vald, val.data(), nnz * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  }
  if (h->mixed) {
    TRY(alloc_fixed(h, &sd.valf, std::max<int64_t>(nnz, 1)));
    sylv::launch_convert<float>(h->stream, nnz, sd.vald, sd.valf);
  }
  CU(cudaStreamSynchronize(h->stream));  // the host vectors go out of scope
  return SYLV_OK;
}

int upload_rhs(sylv_handle* h, Side& sd, const double* C) {
  const int64_t cnt = sd.n * h->s;
  for (int64_t i = 0; i < cnt; ++i)
    if (!std::isfinite(C[i])) return fail(SYLV_ENONFINITE, "non-finite right-hand side entry");
  TRY(alloc_fixed(h, &sd.C, cnt));
  CU(cudaMemcpyAsync(sd.C, C, cnt * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  TRY(alloc_fixed(h, &sd.RQR, 64));
  TRY(alloc_fixed(h, &sd.R1, 64));
  TRY(alloc_fixed(h, &sd.Rinv, 64));
  TRY(alloc_fixed(h, (double**)&sd.RinvT, 64));
  return SYLV_OK;
}

int nsides(const sylv_handle* h) { return h->lyap ? 1 : 2; }

cudaEvent_t prof_event(sylv_handle* h) {
  Prof& p = h->prof;
  if (p.used == p.pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    p.pool.push_back(e);
  }
  return p.pool[p.used++];
}

cudaEvent_t prof_begin(sylv_handle* h) {
  if (!h->prof.on) return nullptr;
  cudaEvent_t a = prof_event(h);
  if (a) cudaEventRecord(a, h->prof_stream ? h->prof_stream : h->stream);
  return a;
}

void prof_end(sylv_handle* h, int cls, double bytes, double flops, cudaEvent_t a) {
  if (!h->prof.on || !a) return;
  cudaEvent_t b = prof_event(h);
  if (!b) return;
  cudaEventRecord(b, h->prof_stream ? h->prof_stream : h->stream);
  h->prof.recs.push_back({cls, h->prof.cur_k, a, b, bytes, flops});
}

void prof_reset(sylv_handle* h) {
  Prof& p = h->prof;
  p.on = h->opt.profile != 0;
  p.used = 0;
  p.recs.clear();
  p.flushed = 0;
  p.cur_k = -1;
  p.valid = false;
  for (int i = 0; i < KC_NUM; ++i) {
    p.launches[i] = 0;
    p.ms[i] = p.bytes[i] = p.flops[i] = 0.0;
  }
}

// After the final synchronisation: sum the launches that belong to completed iterations.
void prof_finish(sylv_handle* h, int iters) {
  Prof& p = h->prof;
  if (!p.on) return;
  for (size_t i = p.flushed; i < p.recs.size(); ++i) {
    const auto& r = p.recs[i];
    if (r.k >= iters) continue;  // enqueued after the stop: no-op launches
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    p.launches[r.cls] += 1;
    p.ms[r.cls] += ms;
    p.bytes[r.cls] += r.bytes;
    p.flops[r.cls] += r.flops;
  }
  p.flushed = p.recs.size();
  p.valid = true;
}

#define PROF(h, cls, bytes, flops, stmt)            \
  do {                                              \
    cudaEvent_t prof_a_ = prof_begin(h);            \
    stmt;                                           \
    prof_end((h), (cls), (bytes), (flops), prof_a_); \
  } while (0)

// Device buffers sized for `maxb` basis blocks per side.
// Order r from which the small Sylvester operator runs on the tensor cores (option small_gemm = 0).
constexpr int kOzakiMinR = 448;  // measured crossover with the CUDA-core float64 kernel

int ensure_capacity(sylv_handle* h, int method, int maxb, int hist_need) {
  const bool want_oz = arnoldi_method(method) && h->opt.small_gemm != 1 && (int64_t)maxb * h->s >= kOzakiMinR;
  // float64 Arnoldi bases: Gram products and updates on the tensor cores unless basis_gemm = 1
  const bool want_ob = !h->mixed && arnoldi_method(method) && h->opt.basis_gemm != 1;
  if (h->maxb >= maxb && h->hist_cap >= hist_need && h->cap_method != M_NONE && (!want_oz || h->oz_scratch) &&
      (!want_ob || h->side[0].ob.G || h->ob_unavailable) &&
      ((method != M_CGS && method != M_GPBICG) || h->Uh) && (method != M_GPBICG || h->gW))
    return SYLV_OK;
  free_solve(h);
  const int64_t s = h->s;
  const size_t fsz = h->mixed ? sizeof(float) : sizeof(double);
  const int64_t ldh = (int64_t)maxb * s;
  h->lds = ldh;
  for (int i = 0; i < nsides(h); ++i) {
    Side& sd = h->side[i];
    TRY(dev_alloc(h, h->solve_allocs, &sd.V, (size_t)maxb * sd.n * s * fsz));
    TRY(alloc_solve(h, &sd.H, (size_t)(ldh * ldh)));
  }
  const size_t l2 = (size_t)(h->lds * h->lds);
  TRY(alloc_solve(h, &h->Xh, l2));
  TRY(alloc_solve(h, &h->Rh, l2));
  TRY(alloc_solve(h, &h->Ph, l2));
  TRY(alloc_solve(h, &h->Qh, l2));
  TRY(alloc_solve(h, &h->Sh, l2));
  TRY(alloc_solve(h, &h->Th, l2));
  if (method == M_CGS || method == M_GPBICG) TRY(alloc_solve(h, &h->Uh, l2));
  if (method == M_GPBICG) {
    TRY(alloc_solve(h, &h->gW, l2));
    TRY(alloc_solve(h, &h->gZ, l2));
    TRY(alloc_solve(h, &h->gTp, l2));
    TRY(alloc_solve(h, &h->gY, l2));
    TRY(alloc_solve(h, &h->gPart, (size_t)5 * sylv::GP_ZETA_CTAS));
  }
  TRY(alloc_solve(h, &h->Rt, 64));
  TRY(alloc_solve(h, &h->hist, (size_t)hist_need));
  // Gram partials: at most 2*SMs CTAs x (maxb * s * s)
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  TRY(alloc_solve(h, &h->spart, (size_t)(4 * sms) * 64));
  TRY(alloc_solve(h, &h->spart2, (size_t)(4 * sms) * 64));
  for (int i = 0; i < nsides(h); ++i) {
    TRY(alloc_solve(h, &h->gpart_s[i], (size_t)(4 * sms) * maxb * s * s));
    TRY(alloc_solve(h, &h->spart_s[i], (size_t)(4 * sms) * 64));
    TRY(alloc_solve(h, &h->spart2_s[i], (size_t)(4 * sms) * 64));
    TRY(alloc_solve(h, &h->Hc_s[i], (size_t)maxb * s * s));
  }
  const int64_t gtiles = (h->lds + 31) / 32;
  const size_t psz = std::max<size_t>((size_t)((h->lds + sylv::NT - 1) / sylv::NT) * h->lds, 2 * gtiles * gtiles) + 64;
  TRY(alloc_solve(h, &h->psmall, psz));
  if (h->mixed) {
    TRY(alloc_solve(h, &h->Hs, l2));
    if (!h->lyap) TRY(alloc_solve(h, &h->Gs, l2));
    TRY(alloc_solve(h, &h->Zs, l2));
  }
  // tensor-core small products: the dense (Arnoldi) operator only, once it is large enough
  if (want_oz) {
    if (!sylv::ozaki_setup()) return fail(SYLV_ECUDA, "tensor-core kernel setup");
    unsigned char* p = nullptr;
    TRY(alloc_solve(h, &p, sylv::ozaki_scratch_bytes((int)ldh)));
    h->oz_scratch = p;
  }
  // digit planes of the float64 Arnoldi bases (twice 10 bytes per basis element per side);
  // zero-filled once, so that padding rows and columns hold finite digits
  h->ob_unavailable = false;
  if (want_ob) {
    if (!sylv::ob_setup()) return fail(SYLV_ECUDA, "tensor-core basis kernel setup");
    const std::string err0 = g_err;
    for (int i = 0; i < nsides(h); ++i) {
      Side& sd = h->side[i];
      const size_t bytes = sylv::ob_side_bytes(sd.n, (int)ldh, (int)s);
      void* p = nullptr;
      const int rc = dev_alloc(h, h->solve_allocs, &p, bytes);
      if (rc != SYLV_OK) {
        if (rc != SYLV_ENOMEM || h->opt.basis_gemm == 2) return rc;
        // not enough device memory: the CUDA-core float64 kernels run instead
        for (int j = 0; j < nsides(h); ++j) h->side[j].ob = sylv::ObSide{};
        h->ob_unavailable = true;
        g_err = err0;
        break;
      }
      CU(cudaMemsetAsync(p, 0, bytes, h->stream));
      sylv::ob_carve(p, sd.n, (int)ldh, (int)s, sd.ob);
    }
  }
  h->maxb = maxb;
  h->hist_cap = hist_need;
  h->cap_method = method;
  return SYLV_OK;
}

template <typename T>
const T* op_val(const Side& sd);
template <>
const double* op_val<double>(const Side& sd) { return sd.vald; }
template <>
const float* op_val<float>(const Side& sd) { return sd.valf; }

double deflate_tol(const sylv_handle* h) {
  if (h->opt.deflate_tol > 0) return h->opt.deflate_tol;
  return h->mixed ? 1e-6 : 1e-12;
}

// Thin QR of C (CholQR2) into block 0; R -> sd.RQR.
template <typename T>
void setup_qr(sylv_handle* h, int si) {
  Side& sd = h->side[si];
  const int s = (int)h->s;
  T* V0 = (T*)sd.V;
  // tensor-core basis: the column maxima are combined from zero (the last scale fills [0, 8))
  if (sd.ob.G) cudaMemsetAsync(sd.ob.mx, 0, 16 * sizeof(unsigned long long), h->stream);
  sylv::launch_pack<T>(h->stream, sd.n, s, sd.C, V0);
  int nc = sylv::launch_selfgram<T>(h->stream, h->st, sd.n, s, V0, h->spart);
  sylv::CholArgs a{};
  a.side = si;
  a.s = s;
  a.delta = deflate_tol(h);
  a.R1 = sd.R1;
  a.Rinv = sd.Rinv;
  a.RinvT = sd.RinvT;
  a.factor_is_float = h->mixed ? 1 : 0;
  a.setup = 1;
  a.pass = 1;
  a.ldh = 0;
  nc = sylv::launch_cholscale<T>(h->stream, h->st, h->spart, nc, a, sd.n, V0, h->spart2, nullptr);
  a.pass = 2;
  a.Rout = sd.RQR;
  sylv::launch_cholscale<T>(h->stream, h->st, h->spart2, nc, a, sd.n, V0, nullptr, sd.ob.G ? sd.ob.mx : nullptr);
  if (sd.ob.G) sylv::launch_ob_split_basis(h->stream, h->st, sd.n, s, (const double*)V0, 0, sd.ob);
}

// Digit planes of the basis in the second BCGS2 update Y2 = Y1 - V H2.  Y1 is already orthogonal
// to V up to rounding, so |H2| ~ eps ||Y||: the basis's top two digit planes (22 bits) leave an
// error below 2^-23 of that correction, far under the float64 rounding of Y2 -- the pass reads
// 4 bytes per basis element instead of 10.  The Gram products and the first update use all 5.
constexpr int kReorthPlanes = 2;

// One block Lanczos (lanczos=true) or BCGS2 block Arnoldi step on side si:
// from blocks 0..q build block q+1 and column block q of H (eq. 3.4).
template <typename T>
void basis_step(sylv_handle* h, int si, int q, bool lanczos) {
  Side& sd = h->side[si];
  const int s = (int)h->s;
  const int64_t n = sd.n, bstride = n * s, ldh = h->lds;
  const double b = (double)sizeof(T);
  const double ns = (double)n * s;
  T* V = (T*)sd.V;
  T* Vq = V + (int64_t)q * bstride;
  T* Y = V + (int64_t)(q + 1) * bstride;
  cudaStream_t st = h->sbas[si];
  h->prof_stream = st;
  double* gpart = h->gpart_s[si];
  double* spart = h->spart_s[si];
  double* Hc = h->Hc_s[si];
  int nc;
  // algorithmic bytes: CSR once, gathered block once, result once (+ V_{j-1} for Lanczos)
  const double spmm_bytes = (double)sd.nnz * (4.0 + b) + 4.0 * (n + 1) + 2.0 * ns * b + (lanczos && q >= 1 ? ns * b : 0.0);
  const double spmm_flops = 2.0 * sd.nnz * s + (lanczos && q >= 1 ? 2.0 * ns * s : 0.0);
  const int nb = lanczos ? 1 : q + 1;
  const T* Vfirst = lanczos ? Vq : V;
  // float64 Arnoldi: the Gram products and updates on the tensor cores, on the digit planes
  const bool ob = !lanczos && sd.ob.G != nullptr;
  const double gram_bytes = ns * b * (nb + 1), gram_flops = 2.0 * ns * nb * s;
  const double upd_bytes = ns * b * (nb + 2), upd_flops = 2.0 * ns * nb * s;
  if (lanczos) {
    const T* Vprev = q >= 1 ? V + (int64_t)(q - 1) * bstride : nullptr;
    const double* M = q >= 1 ? sd.H + (int64_t)(q - 1) * s + (int64_t)q * s * ldh : nullptr;
    PROF(h, KC_SPMM, spmm_bytes, spmm_flops,
         sylv::launch_spmm<T>(st, h->st, n, s, sd.rp, sd.ci, op_val<T>(sd), Vq, Y, Vprev, M, ldh));
  } else {
    PROF(h, KC_SPMM, spmm_bytes, spmm_flops,
         sylv::launch_spmm<T>(st, h->st, n, s, sd.rp, sd.ci, op_val<T>(sd), Vq, Y, nullptr, nullptr, 0,
                              ob ? sd.ob.mx + 8 : nullptr));
  }
  const int passes = lanczos ? 1 : 2;  // block Lanczos: one projection; Arnoldi: BCGS2
  const int js = nb * s;
  for (int pass = 0; pass < passes; ++pass) {
    const bool last = pass == passes - 1;
    if (ob) {
      double* Yd = (double*)Y;
      PROF(h, KC_GRAM, gram_bytes, gram_flops, nc = sylv::launch_ob_gram(st, h->st, n, s, js, Yd, sd.ob, gpart));
      // the reduction's last CTA also writes the coefficient digits for the update
      PROF(h, KC_REDUCE, (double)nc * nb * s * s * 8.0, (double)nc * nb * s * s,
           sylv::launch_ob_reduce_H(st, h->st, si, gpart, nc, nb, s, sd.H, ldh, 0, (int64_t)q * s, Hc, pass == 1,
                                    sd.ob));
      PROF(h, KC_UPDATE, upd_bytes, upd_flops + (last ? ns * s : 0.0),
           nc = sylv::launch_ob_update(st, h->st, n, s, js, Hc, Yd, sd.ob, last ? spart : nullptr, !last,
                                       last ? kReorthPlanes : 5, true));
      continue;
    }
    PROF(h, KC_GRAM, gram_bytes, gram_flops, nc = sylv::launch_gram<T>(st, h->st, n, s, Vfirst, bstride, nb, Y, gpart));
    PROF(h, KC_REDUCE, (double)nc * nb * s * s * 8.0, (double)nc * nb * s * s,
         sylv::launch_reduce_H(st, h->st, gpart, nc, nb, s, sd.H, ldh, lanczos ? (int64_t)q * s : 0,
                               (int64_t)q * s, Hc, pass == 1, sizeof(T) == 4));
    PROF(h, KC_UPDATE, upd_bytes, upd_flops + (last ? ns * s : 0.0),
         nc = sylv::launch_update<T>(st, h->st, n, s, Vfirst, bstride, nb, Hc, Y, last ? spart : nullptr));
  }
  sylv::CholArgs a{};
  a.side = si;
  a.s = s;
  a.delta = deflate_tol(h);
  a.Hcol = sd.H + (int64_t)q * s * ldh;
  a.ldh = ldh;
  a.hrows = (int64_t)(q + 1) * s;
  a.R1 = sd.R1;
  a.Rinv = sd.Rinv;
  a.RinvT = sd.RinvT;
  a.factor_is_float = h->mixed ? 1 : 0;
  a.pass = 1;
  // each CholQR pass is one launch: Cholesky of the s x s Gram (in every CTA) and the scaling
  double* spart2 = h->spart2_s[si];
  PROF(h, KC_SCALE, 2.0 * ns * b, ns * (s + 1) + ns * s,
       nc = sylv::launch_cholscale<T>(st, h->st, spart, nc, a, n, Y, spart2, nullptr));
  a.pass = 2;
  a.Hsub = sd.H + (int64_t)(q + 1) * s + (int64_t)q * s * ldh;
  a.Hsup = lanczos ? sd.H + (int64_t)q * s + (int64_t)(q + 1) * s * ldh : nullptr;
  PROF(h, KC_SCALE, 2.0 * ns * b, ns * (s + 1),
       sylv::launch_cholscale<T>(st, h->st, spart2, nc, a, n, Y, nullptr, ob ? sd.ob.mx : nullptr));
  if (ob)
    PROF(h, KC_BSPLIT, 2.0 * ns * b + 20.0 * ns, 0.0,
         sylv::launch_ob_split_basis(st, h->st, n, s, (const double*)Y, (q + 1) * s, sd.ob));
  h->prof_stream = nullptr;
}

sylv::SmallCtx small_ctx(sylv_handle* h) {
  sylv::SmallCtx c{};
  c.st = h->st;
  c.hist = h->hist;
  c.s = (int)h->s;
  c.lds = h->lds;
  c.Xh = h->Xh;
  c.Rh = h->Rh;
  c.Ph = h->Ph;
  c.Qh = h->Qh;
  c.Sh = h->Sh;
  c.Th = h->Th;
  c.Uh = h->Uh;
  c.gW = h->gW;
  c.gZ = h->gZ;
  c.gTp = h->gTp;
  c.gY = h->gY;
  c.gPart = h->gPart;
  c.Rt = h->Rt;
  c.H = h->side[0].H;
  c.G = h->lyap ? h->side[0].H : h->side[1].H;
  c.ldh = h->lds;
  c.partials = h->psmall;
  c.lyapunov = h->lyap ? 1 : 0;
  c.df_small = h->mixed ? 1 : 0;  // mixed mode: double-float small products (2^-48), FP64 mode: FP64
  c.Hs = h->Hs;
  c.Gs = h->lyap ? h->Hs : h->Gs;
  c.Zs = h->Zs;
  c.split_cols = &h->split_cols;
  c.oz_scratch = h->oz_scratch;
  c.oz_min_r = h->opt.small_gemm == 2 ? 1 : kOzakiMinR;
  return c;
}

// Copy the device status to pinned slot `slot` and record its event.
int post_status(sylv_handle* h, int slot) {
  CU(cudaMemcpyAsync(&h->st_host[slot], h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaEventRecord(h->ev[slot], h->stream));
  return SYLV_OK;
}

int wait_status(sylv_handle* h, int slot, double deadline) {
  for (;;) {
    cudaError_t e = cudaEventQuery(h->ev[slot]);
    if (e == cudaSuccess) return SYLV_OK;
    if (e != cudaErrorNotReady) return fail(SYLV_ECUDA, std::string("solve: ") + cudaGetErrorString(e));
    if (now_s() > deadline) return fail(SYLV_ETIMEOUT, "device did not finish within the timeout");
    std::this_thread::yield();
  }
}

int ensure_streams(sylv_handle* h) {
  if (h->sbas[0]) return SYLV_OK;
  // The larger side's basis chain is the solve's critical path (its HBM-bound Gram and updates
  // take the most time); its stream gets the highest priority, so that the other side's kernels
  // fill the SMs its latency-bound kernels (CholQR, digit splits, reductions) leave idle.
  int prio_lo = 0, prio_hi = 0;
  CU(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
  const int big = (!h->lyap && h->side[1].n > h->side[0].n) ? 1 : 0;
  for (int i = 0; i < 2; ++i)
    CU(cudaStreamCreateWithPriority(&h->sbas[i], cudaStreamNonBlocking, i == big ? prio_hi : prio_lo));
  CU(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  for (auto& pr : h->ev_bas)
    for (auto& e : pr) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  for (auto& e : h->ev_small) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return SYLV_OK;
}

// The bases run at most this many iterations ahead of the small side.
constexpr int kBasisLag = 2;

template <typename T>
int run_inner(sylv_handle* h, int method, double tol, int maxit, sylv_info* info) {
  const double t0 = now_s();
  const double deadline = t0 + (h->opt.timeout_s > 0 ? h->opt.timeout_s : 3600.0);
  if (!(tol >= 0.0) || maxit < 0) return fail(SYLV_EINVAL, "tol must be >= 0 and maxit >= 0");
  // CG: V_{k+2} in iteration k; CR: one step ahead (L(R_{k+1}) needs V_{k+3}); Arnoldi: two per iteration
  const int maxb = std::max(2, method == M_CG ? maxit + 1 : method == M_CR ? maxit + 2 : 2 * maxit + 1);
  TRY(ensure_capacity(h, method, maxb, maxit + 1));
  h->cert_valid = false;  // the bases change
  h->cert_failed = false;
  const int s = (int)h->s;
  cudaStream_t strm = h->stream;
  CU(cudaMemsetAsync(h->st, 0, sizeof(DevState), strm));
  const size_t l2 = (size_t)(h->lds * h->lds) * sizeof(double);
  for (double* p : {h->Xh, h->Rh, h->Ph, h->Qh, h->Sh, h->Th, h->Uh, h->gW, h->gZ, h->gTp, h->gY})
    if (p) CU(cudaMemsetAsync(p, 0, l2, strm));
  for (int i = 0; i < nsides(h); ++i) CU(cudaMemsetAsync(h->side[i].H, 0, l2, strm));
  if (h->mixed) {  // split copies of H, G follow H's zero fill
    CU(cudaMemsetAsync(h->Hs, 0, l2, strm));
    if (!h->lyap) CU(cudaMemsetAsync(h->Gs, 0, l2, strm));
  }
  h->split_cols = 0;
  prof_reset(h);
  const int64_t launches0 = sylv::launch_counter();
  for (int i = 0; i < nsides(h); ++i) {
    PROF(h, KC_SETUP, 0.0, 0.0, setup_qr<T>(h, i));
  }
  sylv::SmallCtx c = small_ctx(h);
  const Side& sA = h->side[0];
  const Side& sB = h->side[h->lyap ? 0 : 1];
  sylv::launch_init_small(strm, c, sA.RQR, sB.RQR, tol, method == M_CGS);
  CU(cudaGetLastError());
  const int poll = h->opt.poll_every > 0 ? h->opt.poll_every : 8;
  int slot = 0, pending = -1;
  bool stopped = false;
  TRY(ensure_streams(h));
  const int ns_ = nsides(h);
  // concurrent bases only where they pay (measured): memory-bound basis sweeps -- the mixed
  // mode's, and the float64 Arnoldi bases on the tensor cores (517 vs 660 ms per benchmarked
  // solve) -- leave room for the other side's and the small side's kernels; the CUDA-core
  // float64 kernels all compete for the FP64 pipe
  const int mode = h->opt.stream_mode;
  const bool tensor_basis = arnoldi_method(method) && h->side[0].ob.G != nullptr;
  const bool concurrent = mode == 2 || (mode == 0 && (h->mixed || tensor_basis));
  // On every exit path (an early return after SYLV_ETIMEOUT or a CUDA error included) the main
  // stream waits for the basis streams, so that the next call on the handle, which starts on the
  // main stream, is ordered after every kernel this solve enqueued; the handle keeps owning its
  // two streams.
  struct RestoreBasisStreams {
    sylv_handle* h;
    cudaStream_t a, b;
    ~RestoreBasisStreams() {
      for (int i = 0; i < 2; ++i)
        if (h->sbas[i] != nullptr && h->sbas[i] != h->stream && h->ev_bas[i][0] != nullptr &&
            cudaEventRecord(h->ev_bas[i][0], h->sbas[i]) == cudaSuccess)
          cudaStreamWaitEvent(h->stream, h->ev_bas[i][0], 0);
      h->sbas[0] = a;
      h->sbas[1] = b;
    }
  } restore{h, h->sbas[0], h->sbas[1]};
  if (!concurrent) h->sbas[0] = h->sbas[1] = strm;
  // fork: the basis streams start after the setup on the main stream
  CU(cudaEventRecord(h->ev_fork, strm));
  for (int i = 0; i < ns_; ++i) CU(cudaStreamWaitEvent(h->sbas[i], h->ev_fork, 0));
  const double e8 = 8.0;
  auto basis_wait_small = [&](int k) -> int {  // throttle: basis of iteration k after small side of k - lag
    if (k < kBasisLag) return SYLV_OK;
    for (int i = 0; i < ns_; ++i) CU(cudaStreamWaitEvent(h->sbas[i], h->ev_small[(k - kBasisLag) % 8], 0));
    return SYLV_OK;
  };
  auto small_wait_basis = [&](int which) -> int {  // small side after basis event `which` of every side
    for (int i = 0; i < ns_; ++i) {
      CU(cudaEventRecord(h->ev_bas[i][which], h->sbas[i]));
      CU(cudaStreamWaitEvent(strm, h->ev_bas[i][which], 0));
    }
    return SYLV_OK;
  };
  if (method == M_CR) {  // L(R_0) needs V_2: one Lanczos step, the operator on R^_0, P^_0 = R^_0, alpha
    basis_step<T>(h, 0, 0, true);
    if (!h->lyap) basis_step<T>(h, 1, 0, true);
    TRY(small_wait_basis(0));
    const double r2 = 4.0 * s * s;
    if (h->lyap) {
      PROF(h, KC_SMALL_OP, e8 * 2.0 * r2, r2, sylv::launch_cr_op(strm, c, 1, s, true));
      PROF(h, KC_SMALL_OP, e8 * 3.0 * r2, r2, sylv::launch_cr_op(strm, c, 2, s, true));
    } else {
      PROF(h, KC_SMALL_OP, e8 * 2.0 * r2, 2.0 * r2, sylv::launch_cr_op(strm, c, 0, s, true));
    }
    PROF(h, KC_SMALL_ELEM, e8 * 5.0 * r2, 5.0 * r2, sylv::launch_cr_p(strm, c, 2 * s));
  }
  for (int k = 0; k < maxit && !stopped; ++k) {
    h->prof.cur_k = k;
    TRY(basis_wait_small(k));
    if (method == M_CR) {  // the update and test first; then L(R_{k+1}) on V_{k+3}
      const int r = (k + 1) * s, rp = r + s, rpp = rp + s;
      const double q2 = (double)rp * rp, t2 = (double)rpp * rpp;
      PROF(h, KC_SMALL_ELEM, e8 * 6.0 * q2, 4.0 * q2, sylv::launch_cg_update(strm, c, k, r, true));
      basis_step<T>(h, 0, k + 1, true);
      if (!h->lyap) basis_step<T>(h, 1, k + 1, true);
      TRY(small_wait_basis(0));
      const double opflops = 2.0 * 2.0 * t2 * 3.0 * s;
      if (h->lyap) {
        PROF(h, KC_SMALL_OP, e8 * (2.0 * t2), opflops / 2, sylv::launch_cr_op(strm, c, 1, rp, false));
        PROF(h, KC_SMALL_OP, e8 * (3.0 * t2), t2, sylv::launch_cr_op(strm, c, 2, rp, false));
      } else {
        PROF(h, KC_SMALL_OP, e8 * (2.0 * t2), opflops, sylv::launch_cr_op(strm, c, 0, rp, false));
      }
      PROF(h, KC_SMALL_ELEM, e8 * 5.0 * t2, 5.0 * t2, sylv::launch_cr_p(strm, c, rpp));
    } else if (method == M_CG) {
      basis_step<T>(h, 0, k, true);
      if (!h->lyap) basis_step<T>(h, 1, k, true);
      TRY(small_wait_basis(0));
      const int r = (k + 1) * s, rp = r + s;
      const double r2 = (double)rp * rp;
      const double opflops = 2.0 * 2.0 * r2 * 3.0 * s;
      if (h->lyap) {
        PROF(h, KC_SMALL_OP, e8 * (2.0 * r2), opflops / 2, sylv::launch_cg_q(strm, c, 1, r));
        PROF(h, KC_SMALL_OP, e8 * (3.0 * r2), r2, sylv::launch_cg_q(strm, c, 2, r));
      } else {
        PROF(h, KC_SMALL_OP, e8 * (2.0 * r2), opflops, sylv::launch_cg_q(strm, c, 0, r));
      }
      PROF(h, KC_SMALL_ELEM, e8 * 6.0 * r2, 4.0 * r2, sylv::launch_cg_update(strm, c, k, r));
      PROF(h, KC_SMALL_ELEM, e8 * 3.0 * r2, 2.0 * r2, sylv::launch_cg_p(strm, c, rp));
    } else if (method == M_BICG) {
      const int r1 = (2 * k + 1) * s, rp = r1 + s, rpp = rp + s;
      const double q2 = (double)rp * rp, t2 = (double)rpp * rpp;
      basis_step<T>(h, 0, 2 * k, false);
      basis_step<T>(h, 1, 2 * k, false);
      TRY(small_wait_basis(0));
      PROF(h, KC_SMALL_GEMM, e8 * (3.0 * (double)r1 * r1 + q2), sylv::sylv_gemm_flops(r1, s),
           sylv::launch_sylv_gemm(strm, c, r1, c.Ph, c.Qh, false));
      PROF(h, KC_SMALL_ELEM, 0.0, 0.0, sylv::launch_bicg_alpha(strm, c));
      PROF(h, KC_SMALL_ELEM, e8 * 3.0 * q2, 2.0 * q2, sylv::launch_bicg_s(strm, c, rp));
      basis_step<T>(h, 0, 2 * k + 1, false);
      basis_step<T>(h, 1, 2 * k + 1, false);
      TRY(small_wait_basis(1));
      PROF(h, KC_SMALL_GEMM, e8 * (3.0 * q2 + t2), sylv::sylv_gemm_flops(rp, s) + 4.0 * t2,
           sylv::launch_sylv_gemm(strm, c, rp, c.Sh, c.Th, true));
      PROF(h, KC_SMALL_ELEM, e8 * (4.0 * q2 + 3.0 * t2), 4.0 * q2 + 4.0 * t2,
           sylv::launch_bicg_update(strm, c, k, rp, rpp));
      PROF(h, KC_SMALL_ELEM, e8 * 4.0 * t2, 4.0 * t2, sylv::launch_bicg_p(strm, c, rpp));
    } else if (method == M_GPBICG) {  // the same bases and operator, the GPBiCG recurrences
      const int e1 = (2 * k + 1) * s, e2 = e1 + s, e3 = e2 + s;
      const double q1 = (double)e1 * e1, q2 = (double)e2 * e2, q3 = (double)e3 * e3;
      PROF(h, KC_SMALL_ELEM, e8 * 4.0 * q1, 3.0 * q1, sylv::launch_gp_p(strm, c, e1));
      basis_step<T>(h, 0, 2 * k, false);
      basis_step<T>(h, 1, 2 * k, false);
      TRY(small_wait_basis(0));
      PROF(h, KC_SMALL_GEMM, e8 * (3.0 * q1 + q2), sylv::sylv_gemm_flops(e1, s),
           sylv::launch_sylv_gemm(strm, c, e1, c.Ph, c.Qh, false));  // L(P)^
      PROF(h, KC_SMALL_ELEM, 0.0, 0.0, sylv::launch_bicg_alpha(strm, c));
      PROF(h, KC_SMALL_ELEM, e8 * 6.0 * q2, 6.0 * q2, sylv::launch_gp_ty(strm, c, e2));
      basis_step<T>(h, 0, 2 * k + 1, false);
      basis_step<T>(h, 1, 2 * k + 1, false);
      TRY(small_wait_basis(1));
      PROF(h, KC_SMALL_GEMM, e8 * (3.0 * q2 + q3), sylv::sylv_gemm_flops(e2, s),
           sylv::launch_sylv_gemm(strm, c, e2, c.Th, c.Sh, false));  // L(T)^
      PROF(h, KC_SMALL_ELEM, e8 * (3.0 * q2 + q3), 8.0 * q2 + 2.0 * q3, sylv::launch_gp_zeta(strm, c, k, e2));
      PROF(h, KC_SMALL_ELEM, e8 * (10.0 * q2 + 4.0 * q3), 12.0 * q2 + 6.0 * q3, sylv::launch_gp_update(strm, c, k, e2));
      PROF(h, KC_SMALL_ELEM, e8 * 5.0 * q3, 2.0 * q3, sylv::launch_gp_w(strm, c, e3));
    } else {  // M_CGS: the same bases and operator, the CGS recurrences on the small side
      const int r1 = (2 * k + 1) * s, rp = r1 + s, rpp = rp + s;
      const double q2 = (double)rp * rp, t2 = (double)rpp * rpp;
      basis_step<T>(h, 0, 2 * k, false);
      basis_step<T>(h, 1, 2 * k, false);
      TRY(small_wait_basis(0));
      PROF(h, KC_SMALL_GEMM, e8 * (3.0 * (double)r1 * r1 + q2), sylv::sylv_gemm_flops(r1, s),
           sylv::launch_sylv_gemm(strm, c, r1, c.Ph, c.Qh, false));  // V^ = L(P^)
      PROF(h, KC_SMALL_ELEM, 0.0, 0.0, sylv::launch_bicg_alpha(strm, c));
      PROF(h, KC_SMALL_ELEM, e8 * 6.0 * q2, 4.0 * q2, sylv::launch_cgs_q(strm, c, rp));
      basis_step<T>(h, 0, 2 * k + 1, false);
      basis_step<T>(h, 1, 2 * k + 1, false);
      TRY(small_wait_basis(1));
      PROF(h, KC_SMALL_GEMM, e8 * (3.0 * q2 + t2), sylv::sylv_gemm_flops(rp, s),
           sylv::launch_sylv_gemm(strm, c, rp, c.Th, c.Sh, false));  // T^ = L(W^)
      PROF(h, KC_SMALL_ELEM, e8 * 3.0 * t2, 4.0 * t2, sylv::launch_cgs_update(strm, c, k, rpp));
      PROF(h, KC_SMALL_ELEM, e8 * 5.0 * t2, 5.0 * t2, sylv::launch_cgs_p(strm, c, rpp));
    }
    CU(cudaEventRecord(h->ev_small[k % 8], strm));
    if ((k + 1) % poll == 0 && k + 1 < maxit) {
      CU(cudaGetLastError());
      TRY(post_status(h, slot));
      if (pending >= 0) {
        TRY(wait_status(h, pending, deadline));
        if (h->st_host[pending].status != sylv::ST_RUNNING) stopped = true;
      }
      pending = slot;
      slot ^= 1;
    }
  }
  CU(cudaGetLastError());
  for (int i = 0; i < ns_; ++i) {  // join the basis streams
    CU(cudaEventRecord(h->ev_bas[i][0], h->sbas[i]));
    CU(cudaStreamWaitEvent(strm, h->ev_bas[i][0], 0));
  }

  TRY(post_status(h, slot));
  TRY(wait_status(h, slot, deadline));
  const DevState& ds = h->st_host[slot];
  prof_finish(h, ds.iters);
  h->method = method;
  h->iters = ds.iters;
  h->width = (int64_t)(lanczos_method(method) ? ds.iters : 2 * ds.iters) * s;
  h->nblocks = lanczos_method(method) ? ds.iters + 1 : 2 * ds.iters + 1;
  int rc;
  switch (ds.status) {
    case sylv::ST_CONVERGED: rc = SYLV_OK; break;
    case sylv::ST_RUNNING: rc = SYLV_ENOTCONV; break;
    case sylv::ST_BREAKDOWN: rc = SYLV_EBREAKDOWN; g_err = "breakdown (site " + std::to_string(ds.breakdown_where) + ")"; break;
    case sylv::ST_WAIT_TIMEOUT: rc = SYLV_ETIMEOUT; g_err = "a device-side wait gave up (site " + std::to_string(ds.breakdown_where) + ")"; break;
    default: rc = SYLV_ENONFINITE; g_err = "non-finite value (site " + std::to_string(ds.breakdown_where) + ")"; break;
  }
  if (maxit == 0 && ds.status == sylv::ST_RUNNING) rc = SYLV_ENOTCONV;
  h->status = rc;
  h->launches = sylv::launch_counter() - launches0;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = rc;
    info->iters = ds.iters;
    info->matvecs = (int64_t)(method == M_CG ? ds.iters : method == M_CR ? ds.iters + 1 : 2 * ds.iters);
    info->width = h->width;
    info->rel_res = ds.r0 > 0 ? ds.rnorm / ds.r0 : 0.0;
    info->true_rel_res = -1.0;
    info->true_rel_bound = -1.0;
    info->solve_ms = (now_s() - t0) * 1e3;
    info->kernel_launches = h->launches;
  }
  return rc;
}


// ------------------------------------------------------------------ float64 true residual
// R = C1 C2^T - A X - X B for X = sum over rounds of V_i X^_i W_i^T is applied to thin
// blocks only, with float64 accumulation:
//   R Om   = C1 (C2^T Om) - A (X Om) - X (B Om)
//   R^T Q  = C2 (C1^T Q)  - X^T (A^T Q) - B^T (X^T Q)
// SYLV_MIXED: a rank-8 randomised range finder with one power iteration gives R ~ Q Z^T with
// Q orthonormal (Q, Z are the right-hand side factors of the next refinement round), and
// ||R||_F^2 = ||Z||_F^2 + ||T||_F^2 with T = (I - Q Q^T) R exactly.  SYLV_FP64: T = R.
//
// Certificate.  A Gaussian block Om (m x k, k = SKT, independent of Q) gives
// ||T Om||_F^2 = sum_i sigma_i(T)^2 X_i with X_i i.i.d. chi-square(k), so ||T Om||^2 / k is
// unbiased for ||T||^2, and for any T and 0 < q < 1 (Chernoff: E exp(-t sum w_i X_i) =
// prod (1 + 2 t w_i)^{-k/2} <= (1 + 2 t sum w_i)^{-k/2})
//   P( ||T Om||^2 <= q k ||T||^2 ) <= (q e^{1-q})^{k/2}.
// With q chosen so that the right side is kCertDelta, the bound
//   ||R||^2 <= ||Z||^2 + ||T Om||^2 / (q k)
// holds with probability at least 1 - kCertDelta over Om, whatever the residual.

constexpr int SKK = 8;  // columns of the sketch blocks
constexpr int SKT = 32;  // columns of the tail probe: SKT / SKK blocks
constexpr double kCertDelta = 1e-4;  // probability that the certified bound fails

// The q of the certificate: the root in (0, 1) of (q e^{1-q})^{SKT/2} = kCertDelta (the left
// side increases on (0, 1)); bisection.
double cert_q() {
  static const double q = [] {
    const double target = std::pow(kCertDelta, 2.0 / SKT);
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid * std::exp(1.0 - mid) < target)
        lo = mid;
      else
        hi = mid;
    }
    return lo;  // the lower end: the bound stays on the safe side
  }();
  return q;
}

double* sk_buf(sylv_handle* h, size_t idx, size_t bytes, int* rc) {
  if (h->sk.size() <= idx) h->sk.resize(idx + 1, {nullptr, 0});
  auto& b = h->sk[idx];
  if (b.second < bytes) {
    // grow geometrically: every cudaFree synchronises the device
    if (b.first) cudaFree(b.first);
    b.first = nullptr;
    b.second = 0;
    bytes = std::max(bytes, (size_t)(1.5 * (double)bytes));
    if (bytes < (1u << 20)) bytes = 1u << 20;
    cudaError_t e = cudaMalloc(&b.first, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *rc = fail(e == cudaErrorMemoryAllocation ? SYLV_ENOMEM : SYLV_ECUDA, "sketch buffer");
      return nullptr;
    }
    b.second = bytes;
  }
  return (double*)b.first;
}

void free_sketch(sylv_handle* h) {
  for (auto& b : h->sk)
    if (b.first) cudaFree(b.first);
  h->sk.clear();
}

void free_subs(sylv_handle* h);

int prepare_residual_ops(sylv_handle* h, const sylv_csr* A, const sylv_csr* B) {
  TRY(upload_operator(h, h->opAt, A, true));
  if (h->lyap)
    h->opB = h->opAt;  // B = A^T
  else
    TRY(upload_operator(h, h->opB, B, false));
  const int s = (int)h->s;
  const int64_t n = h->side[0].n, m = h->lyap ? n : h->side[1].n;
  TRY(alloc_fixed(h, &h->C1rm, n * s));
  TRY(alloc_fixed(h, &h->C2rm, m * s));
  sylv::launch_pack<double>(h->stream, n, s, h->side[0].C, h->C1rm);
  sylv::launch_pack<double>(h->stream, m, s, h->lyap ? h->side[0].C : h->side[1].C, h->C2rm);
  // Gaussian probes: SplitMix64 (Steele, Lea, Flood 2014) + Box-Muller, fixed seed, drawn on the
  // device (counter-based: output i of the stream is a function of i alone)
  const size_t om_count = (size_t)m * (SKK + SKT);  // range block, then the tail probe blocks
  TRY(alloc_fixed(h, &h->Om, om_count));
  sylv::launch_gauss_probes(h->stream, h->Om, om_count, 0x5eedc0de12345678ull);
  CU(cudaGetLastError());
  TRY(alloc_fixed(h, &h->st_sk, 1));
  CU(cudaMallocHost(&h->sk_host, 8 * sizeof(double) + sizeof(DevState)));
  CU(cudaStreamSynchronize(h->stream));
  return SYLV_OK;
}

struct RoundView {
  const void* V;
  const void* W;
  int64_t bsV, bsW;
  int s, nb;
  const double* Xh;
  int64_t lds;
};

std::vector<RoundView> round_views(const sylv_handle* h) {
  std::vector<RoundView> out;
  auto add = [&out](const sylv_handle* x) {  // empty rounds stay (nb = 0) so indices match h->subs
    const Side& a = x->side[0];
    const Side& b = x->side[x->lyap ? 0 : 1];
    out.push_back({a.V, b.V, a.n * x->s, b.n * x->s, (int)x->s, (int)(x->width / x->s), x->Xh, x->lds});
  };
  add(h);
  for (const sylv_handle* sb : h->subs) add(sb);
  return out;
}



// Digit planes of handle x's bases (side 0, side 1) for the certificate's products: the solve's
// own planes where its float64 Arnoldi bases are on the tensor cores; otherwise (float32 bases of
// the mixed mode, or float64 bases on the CUDA cores) built once after the solve, when they take
// at most 30% of the free device memory (the correction solves that follow need the rest), for
// bases of 2^25 elements and more.
// Returns false where none are available (the double-float kernels run instead).
bool cert_planes(sylv_handle* x, const sylv::ObSide** pv, const sylv::ObSide** pw) {
  const int sw = x->lyap ? 0 : 1;
  if (x->opt.cert_gemm == 1) return false;
  if (!x->mixed && x->side[0].ob.G != nullptr && x->side[sw].ob.G != nullptr) {
    *pv = &x->side[0].ob;
    *pw = &x->side[sw].ob;
    return true;
  }
  // small bases (batched instances, tests): the double-float kernels, without the split's launches
  if (x->cert_failed || x->width <= 0 ||
      (x->opt.cert_gemm != 2 && (double)x->side[0].n * (double)x->width < 33554432.0))
    return false;
  if (x->cert_valid && (x->cert_R != x->width || x->cert_V != x->side[0].V)) x->cert_valid = false;
  if (!x->cert_valid) {
    const int s = (int)x->s;
    const int nb = (int)(x->width / s);
    const int R = (int)x->width;
    size_t bytes[2] = {sylv::ob_side_bytes(x->side[0].n, R, s), x->lyap ? 0 : sylv::ob_side_bytes(x->side[1].n, R, s)};
    const size_t need = bytes[0] + bytes[1] + (size_t)R * sizeof(unsigned long long) + 1024;
    if (x->cert_bytes < need) {
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || (double)need > 0.3 * (double)(free_b + x->cert_bytes) ||
          !sylv::ob_setup()) {
        cudaGetLastError();
        x->cert_failed = true;
        return false;
      }
      if (x->cert_mem) cudaFree(x->cert_mem);
      x->cert_mem = nullptr;
      x->cert_bytes = 0;
      if (cudaMalloc(&x->cert_mem, need) != cudaSuccess) {
        cudaGetLastError();
        x->cert_mem = nullptr;
        x->cert_failed = true;
        return false;
      }
      x->cert_bytes = need;
    }
    unsigned char* p = (unsigned char*)x->cert_mem;
    unsigned long long* mx_all = (unsigned long long*)(((uintptr_t)(p + bytes[0] + bytes[1]) + 255) & ~(uintptr_t)255);
    for (int i = 0; i < (x->lyap ? 1 : 2); ++i) {
      Side& sd = x->side[i];
      sylv::ob_carve(p, sd.n, R, s, x->cert_ob[i]);
      // zero-filled, so that padding rows and columns hold finite digits
      if (cudaMemsetAsync(p, 0, bytes[i], x->stream) != cudaSuccess) {
        cudaGetLastError();
        x->cert_failed = true;
        return false;
      }
      sylv::launch_ob_split_bases(x->stream, sd.n, s, nb, sd.V, x->mixed, sd.n * s, mx_all, x->cert_ob[i]);
      p += bytes[i];
    }
    if (x->lyap) x->cert_ob[1] = x->cert_ob[0];
    x->cert_valid = true;
    x->cert_R = x->width;
    x->cert_V = x->side[0].V;
  }
  *pv = &x->cert_ob[0];
  *pw = &x->cert_ob[sw];
  return true;
}

// X^(T) Min for one round whose bases have digit planes (pv: side 0, pw: side 1): the basis
// products on the tensor cores, float64-accurate like the Gram and update of the float64 solve,
// in 8-column pieces of Min; Yout = (first ? 0 : Yout) + the round's term.
int apply_round_ob(sylv_handle* h, bool trans, const double* Min, int k, double* Yout, const RoundView& v,
                   const sylv::ObSide& pv, const sylv::ObSide& pw, bool first) {
  int rc = SYLV_OK;
  const int64_t n = h->side[0].n, m = h->lyap ? n : h->side[1].n;
  const int64_t rows_in = trans ? n : m, rows_out = trans ? m : n;
  const sylv::ObSide& oin0 = trans ? pv : pw;  // Min's side: X^T Min = W X^T (V^T Min)
  const sylv::ObSide& oout0 = trans ? pw : pv;
  const int r = v.nb * v.s;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  constexpr int HW = 8;  // columns per product
  const int64_t nmax = std::max(n, m);
  const int rmax = std::max(pv.rp, pw.rp);
  void* scr = sk_buf(h, 24, sylv::ob_cols_scratch_bytes(nmax, rmax, HW), &rc);
  double* part = sk_buf(h, 25, (size_t)sms * r * HW * sizeof(double), &rc);
  double* H8 = sk_buf(h, 26, (size_t)r * HW * sizeof(double), &rc);
  double* P = sk_buf(h, 0, (size_t)r * k * sizeof(double), &rc);
  double* P2 = sk_buf(h, 1, (size_t)r * k * sizeof(double), &rc);
  if (rc) return rc;
  sylv::ObSide oin = oin0, oout = oout0;
  sylv::ob_cols_carve(scr, nmax, rmax, HW, oin);  // the operand digits: scratch shared by both sides
  oout.YB = oin.YB;
  oout.HB = oin.HB;
  oout.ey = oin.ey;
  oout.eh = oin.eh;
  oout.mx = oin.mx;
  const double fl = 2.0 * (double)r * k;
  for (int c0 = 0; c0 < k; c0 += HW)
    PROF(h, KC_RESID_TSG, (double)rows_in * (r * 8.0 + HW * 8.0), fl / (k / HW) * rows_in,
         sylv::launch_ob_gram_cols(h->stream, h->st_sk, rows_in, HW, r, Min + c0, k, oin, part, P, k, c0));
  PROF(h, KC_RESID_SMALL, 0.0, 2.0 * r * r * k, sylv::launch_small_apply(h->stream, r, k, v.Xh, v.lds, trans, P, P2));
  if (first) CU(cudaMemsetAsync(Yout, 0, (size_t)rows_out * k * sizeof(double), h->stream));
  for (int c0 = 0; c0 < k; c0 += HW) {
    CU(cudaMemcpy2DAsync(H8, HW * sizeof(double), P2 + c0, k * sizeof(double), HW * sizeof(double), r,
                         cudaMemcpyDeviceToDevice, h->stream));
    PROF(h, KC_RESID_TSU, (double)rows_out * (r * 8.0 + 2.0 * HW * 8.0), fl / (k / HW) * rows_out,
         sylv::launch_ob_update_cols(h->stream, h->st_sk, rows_out, HW, r, H8, Yout + c0, k, oout));
  }
  return SYLV_OK;
}

// Yout (rows x k) = X Min (trans = false; Min is m x k) or X^T Min (trans = true; Min is n x k).
template <typename T>
int apply_X(sylv_handle* h, bool trans, const double* Min, int k, double* Yout, size_t from_round = 0) {
  int rc = SYLV_OK;
  const int64_t n = h->side[0].n, m = h->lyap ? n : h->side[1].n;
  const int64_t rows_in = trans ? n : m, rows_out = trans ? m : n;
  auto views = round_views(h);
  if (from_round > 0) views.erase(views.begin(), views.begin() + std::min(from_round, views.size()));
  // rounds whose bases have digit planes run on the tensor cores, the others on the double-float
  // kernels (round 0 is the main solve, round i its i-th correction)
  std::vector<sylv_handle*> hs{h};
  for (sylv_handle* sb : h->subs) hs.push_back(sb);
  if (from_round > 0) hs.erase(hs.begin(), hs.begin() + std::min(from_round, hs.size()));
  int maxw = 1;
  for (auto& v : views) maxw = std::max(maxw, v.nb * v.s);
  const int max_rc = 0;  // launch_tsg picks the row chunks
  double* P = sk_buf(h, 0, (size_t)maxw * k * sizeof(double), &rc);
  double* P2 = sk_buf(h, 1, (size_t)maxw * k * sizeof(double), &rc);
  double* part = sk_buf(h, 2, (size_t)sylv::tsg_partial_elems(maxw, k) * sizeof(double), &rc);
  if (rc) return rc;
  bool first = true;
  for (size_t vi = 0; vi < views.size(); ++vi) {
    const RoundView& v = views[vi];
    if (v.nb <= 0) continue;
    const sylv::ObSide *pv = nullptr, *pw = nullptr;
    if (k % 8 == 0 && vi < hs.size() && cert_planes(hs[vi], &pv, &pw)) {
      TRY(apply_round_ob(h, trans, Min, k, Yout, v, *pv, *pw, first));
      first = false;
      continue;
    }
    const T* Uin = (const T*)(trans ? v.V : v.W);
    const T* Uout = (const T*)(trans ? v.W : v.V);
    const int64_t bsin = trans ? v.bsV : v.bsW, bsout = trans ? v.bsW : v.bsV;
    const int r = v.nb * v.s;
    const double fl = 2.0 * (double)r * k;
    PROF(h, KC_RESID_TSG, (double)rows_in * (r * sizeof(T) + k * 8.0), fl * rows_in,
         sylv::launch_tsg<T>(h->stream, rows_in, Uin, bsin, v.s, v.nb, Min, k, part, max_rc, P));
    PROF(h, KC_RESID_SMALL, 0.0, 2.0 * r * r * k, sylv::launch_small_apply(h->stream, r, k, v.Xh, v.lds, trans, P, P2));
    PROF(h, KC_RESID_TSU, (double)rows_out * (r * sizeof(T) + 2.0 * k * 8.0), fl * rows_out,
         sylv::launch_tsu<T>(h->stream, rows_out, Uout, bsout, v.s, v.nb, P2, k, 1.0, first ? 0.0 : 1.0, Yout));
    first = false;
  }
  if (first) CU(cudaMemsetAsync(Yout, 0, (size_t)rows_out * k * sizeof(double), h->stream));
  return SYLV_OK;
}

// Y (n x 8) = R Om (Om m x 8); X is applied once to the 16 columns [Om | B Om].
// With from_round > 0, Y already holds R_old Om and only the rounds >= from_round
// (the newest correction dX) are applied: R_new Om = R_old Om - (A dX Om + dX B Om).
template <typename T>
int sketch_R(sylv_handle* h, const double* Om, double* Y, size_t from_round = 0) {
  int rc = SYLV_OK;
  const int s = (int)h->s;
  const int64_t n = h->side[0].n, m = h->lyap ? n : h->side[1].n;
  double* G = sk_buf(h, 3, 64 * SKK * sizeof(double), &rc);
  double* part = sk_buf(h, 4, (size_t)sylv::tsg_partial_elems(64, 16) * sizeof(double), &rc);
  double* Tm = sk_buf(h, 5, (size_t)m * SKK * sizeof(double), &rc);
  double* Xa = sk_buf(h, 6, (size_t)n * SKK * sizeof(double), &rc);
  double* Xb = sk_buf(h, 7, (size_t)n * SKK * sizeof(double), &rc);
  double* M16 = sk_buf(h, 20, (size_t)std::max(n, m) * 16 * sizeof(double), &rc);
  double* X16 = sk_buf(h, 21, (size_t)std::max(n, m) * 16 * sizeof(double), &rc);
  if (rc) return rc;
  const Side& Aop = h->side[0];
  sylv::launch_tsg<double>(h->stream, m, h->C2rm, m * s, s, 1, Om, SKK, part, 0, G);       // C2^T Om
  PROF(h, KC_RESID_SPMM, 0.0, 0.0,
       sylv::launch_spmm<double>(h->stream, nullptr, m, SKK, h->opB.rp, h->opB.ci, h->opB.vald, Om, Tm, nullptr,
                                 nullptr, 0));                                               // B Om
  PROF(h, KC_RESID_MISC, 0.0, 0.0, sylv::launch_interleave(h->stream, m, Om, Tm, M16));
  TRY(apply_X<T>(h, false, M16, 16, X16, from_round));                                       // X [Om | B Om]
  sylv::launch_deinterleave(h->stream, n, X16, Xa, Xb);
  if (from_round == 0) {
    sylv::launch_spmm<double>(h->stream, nullptr, n, SKK, Aop.rp, Aop.ci, Aop.vald, Xa, Y, nullptr, nullptr, 0);
    sylv::launch_neg_sum(h->stream, n * SKK, Y, Xb, Y);                                      // -(A X Om + X B Om)
    sylv::launch_lowrank_axpy(h->stream, n, s, SKK, h->C1rm, G, 1.0, Y);                     // + C1 (C2^T Om)
  } else {
    sylv::launch_spmm<double>(h->stream, nullptr, n, SKK, Aop.rp, Aop.ci, Aop.vald, Xa, X16, nullptr, nullptr, 0);
    sylv::launch_neg_sum(h->stream, n * SKK, X16, Xb, X16);                                  // -(A dX Om + dX B Om)
    sylv::launch_axpy(h->stream, n * SKK, 1.0, X16, Y);
  }
  return SYLV_OK;
}

// Z (m x 8) = R^T Q (Q n x 8); X^T is applied once to the 16 columns [A^T Q | Q].
template <typename T>
int sketch_Rt(sylv_handle* h, const double* Q, double* Z) {
  int rc = SYLV_OK;
  const int s = (int)h->s;
  const int64_t n = h->side[0].n, m = h->lyap ? n : h->side[1].n;
  double* G = sk_buf(h, 3, 64 * SKK * sizeof(double), &rc);
  double* part = sk_buf(h, 4, (size_t)sylv::tsg_partial_elems(64, 16) * sizeof(double), &rc);
  double* Tn = sk_buf(h, 8, (size_t)n * SKK * sizeof(double), &rc);
  double* Za = sk_buf(h, 9, (size_t)m * SKK * sizeof(double), &rc);
  double* Zb = sk_buf(h, 10, (size_t)m * SKK * sizeof(double), &rc);
  double* M16 = sk_buf(h, 20, (size_t)std::max(n, m) * 16 * sizeof(double), &rc);
  double* X16 = sk_buf(h, 21, (size_t)std::max(n, m) * 16 * sizeof(double), &rc);
  if (rc) return rc;
  const Side& Bt = h->side[h->lyap ? 0 : 1];  // B^T
  sylv::launch_tsg<double>(h->stream, n, h->C1rm, n * s, s, 1, Q, SKK, part, 0, G);        // C1^T Q
  PROF(h, KC_RESID_SPMM, 0.0, 0.0,
       sylv::launch_spmm<double>(h->stream, nullptr, n, SKK, h->opAt.rp, h->opAt.ci, h->opAt.vald, Q, Tn, nullptr,
                                 nullptr, 0));                                               // A^T Q
  PROF(h, KC_RESID_MISC, 0.0, 0.0, sylv::launch_interleave(h->stream, n, Tn, Q, M16));
  TRY(apply_X<T>(h, true, M16, 16, X16));                                                    // X^T [A^T Q | Q]
  sylv::launch_deinterleave(h->stream, m, X16, Za, Zb);
  sylv::launch_spmm<double>(h->stream, nullptr, m, SKK, Bt.rp, Bt.ci, Bt.vald, Zb, Z, nullptr, nullptr, 0);
  sylv::launch_neg_sum(h->stream, m * SKK, Z, Za, Z);
  sylv::launch_lowrank_axpy(h->stream, m, s, SKK, h->C2rm, G, 1.0, Z);
  return SYLV_OK;
}

// In-place CholQR2 of an n x 8 float64 block (status in st_sk).
void qr8_impl(sylv_handle* h, int64_t n, double* Y, double* Rout);
void qr8(sylv_handle* h, int64_t n, double* Y, double* Rout) {
  PROF(h, KC_RESID_QR, 0.0, 0.0, qr8_impl(h, n, Y, Rout));
}
void qr8_impl(sylv_handle* h, int64_t n, double* Y, double* Rout) {
  double* R1 = Rout + 64;
  double* Rinv = Rout + 128;
  double* RinvT = Rout + 192;
  sylv::CholArgs a{};
  a.side = 0;
  a.s = SKK;
  a.delta = 1e-10;
  a.R1 = R1;
  a.Rinv = Rinv;
  a.RinvT = RinvT;
  a.factor_is_float = 0;
  a.setup = 1;
  a.pass = 1;
  int nc = sylv::launch_selfgram<double>(h->stream, h->st_sk, n, SKK, Y, h->spart);
  nc = sylv::launch_cholscale<double>(h->stream, h->st_sk, h->spart, nc, a, n, Y, h->spart2, nullptr);
  a.pass = 2;
  a.Rout = Rout;
  sylv::launch_cholscale<double>(h->stream, h->st_sk, h->spart2, nc, a, n, Y, nullptr, nullptr);
}

// Enqueues the ||R||_F estimate and its certified bound on h->stream; in SYLV_MIXED also leaves
// Q (n x 8, buffer 11) and Z (m x 8, buffer 12) with R ~ Q Z^T.  sketch_finish waits and reads
// the result.  Host sums: [0] ||Z||^2, [1] ||T Om||^2, [2] ||C1 C2^T||^2, [3] ||R Om||^2.
template <typename T>
int sketch_enqueue(sylv_handle* h) {
  int rc = SYLV_OK;
  const int s = (int)h->s;
  const int64_t n = h->side[0].n, m = h->lyap ? n : h->side[1].n;
  double* Y3 = sk_buf(h, 13, (size_t)n * SKT * sizeof(double), &rc);
  double* sums = sk_buf(h, 15, 8 * sizeof(double), &rc);
  double* part = sk_buf(h, 16, (size_t)256 * sizeof(double) + 64, &rc);
  double* part2 = sk_buf(h, 18, (size_t)sylv::tsg_partial_elems(64, 16) * sizeof(double), &rc);
  // R times the tail probe blocks: persistent across the refinement rounds of one solve and
  // updated with the newest correction only
  double* RO2 = sk_buf(h, 23, (size_t)n * SKT * sizeof(double), &rc);
  if (rc) return rc;
  unsigned int* ticket = (unsigned int*)(part + 256);
  CU(cudaMemsetAsync(h->st_sk, 0, sizeof(DevState), h->stream));
  CU(cudaMemsetAsync(ticket, 0, 16, h->stream));
  CU(cudaMemsetAsync(sums, 0, 8 * sizeof(double), h->stream));
  if (h->cnorm < 0) {
    // ||C1 C2^T||_F^2 = tr((C1^T C1)(C2^T C2))
    double* G1 = sk_buf(h, 19, 128 * sizeof(double), &rc);
    if (rc) return rc;
    sylv::launch_tsg<double>(h->stream, n, h->C1rm, n * s, s, 1, h->C1rm, s, part2, 0, G1);
    sylv::launch_tsg<double>(h->stream, m, h->C2rm, m * s, s, 1, h->C2rm, s, part2, 0, G1 + 64);
    sylv::launch_trace_prod(h->stream, s, G1, G1 + 64, sums + 2);
  }
  const size_t newest = h->subs.size();  // round index of the newest correction (0: none)
  for (int b = 0; b < SKT / SKK; ++b)
    TRY(sketch_R<T>(h, h->Om + (size_t)(1 + b) * m * SKK, RO2 + (size_t)b * n * SKK, newest));
  sylv::launch_sumsq(h->stream, n * SKT, RO2, part, ticket + 2, sums + 3);  // ||R Om||^2
  if (h->mixed) {
    double* Q = sk_buf(h, 11, (size_t)n * SKK * sizeof(double), &rc);
    double* Z = sk_buf(h, 12, (size_t)m * SKK * sizeof(double), &rc);
    double* Rk = sk_buf(h, 14, 256 * sizeof(double), &rc);
    double* P = sk_buf(h, 17, 64 * sizeof(double), &rc);
    double* RO1 = sk_buf(h, 22, (size_t)n * SKK * sizeof(double), &rc);
    if (rc) return rc;
    TRY(sketch_R<T>(h, h->Om, RO1, newest));
    CU(cudaMemcpyAsync(Q, RO1, (size_t)n * SKK * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    qr8(h, n, Q, Rk);
    TRY(sketch_Rt<T>(h, Q, Z));   // Z1 = R^T Q1
    TRY(sketch_R<T>(h, Z, Q));    // power step: Y = R Z1 (a rank-8 range without it is too
    qr8(h, n, Q, Rk);             // poor for the refinement rounds to converge)
    TRY(sketch_Rt<T>(h, Q, Z));   // Z = R^T Q
    // tail probe with the range projected out: T Om = (I - Q Q^T) R Om
    CU(cudaMemcpyAsync(Y3, RO2, (size_t)n * SKT * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    for (int b = 0; b < SKT / SKK; ++b) {
      double* Yb = Y3 + (size_t)b * n * SKK;
      sylv::launch_tsg<double>(h->stream, n, Q, n * SKK, SKK, 1, Yb, SKK, part2, 0, P);
      sylv::launch_tsu<double>(h->stream, n, Q, n * SKK, SKK, 1, P, SKK, -1.0, 1.0, Yb);
    }
    sylv::launch_sumsq(h->stream, m * SKK, Z, part, ticket, sums);
    sylv::launch_sumsq(h->stream, n * SKT, Y3, part, ticket + 1, sums + 1);
  }
  CU(cudaMemcpyAsync(h->sk_host, sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaMemcpyAsync(h->sk_host + 8, h->st_sk, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  return SYLV_OK;
}

// Waits for sketch_enqueue and returns ||R||_F's estimate and certified upper bound.
int sketch_finish(sylv_handle* h, double* est, double* bound, bool* ok) {
  CU(cudaStreamSynchronize(h->stream));
  const double* hs = h->sk_host;
  DevState dst;
  std::memcpy(&dst, h->sk_host + 8, sizeof(DevState));
  if (h->cnorm < 0) h->cnorm = std::sqrt(std::max(0.0, hs[2]));
  if (dst.status == sylv::ST_WAIT_TIMEOUT)
    return fail(SYLV_ETIMEOUT, "a device-side wait of the true-residual certificate gave up (site " +
                                   std::to_string(dst.breakdown_where) + ")");
  const double q = cert_q();
  // the range part is used only when the range finder's CholQR succeeded (R of rank >= 8)
  *ok = h->mixed && dst.status == sylv::ST_RUNNING;
  const double z2 = *ok ? hs[0] : 0.0, t2 = *ok ? hs[1] : hs[3];
  *est = std::sqrt(z2 + t2 / SKT);
  *bound = std::sqrt(z2 + t2 / (q * SKT));
  return SYLV_OK;
}

template <typename T>
int sketch(sylv_handle* h, double* est, double* bound, bool* ok) {
  TRY(sketch_enqueue<T>(h));
  return sketch_finish(h, est, bound, ok);
}

// A correction solve A dX + dX B = Q Z^T on the same operators (s = 8).
int make_sub(sylv_handle* P, sylv_handle** out) {
  *out = nullptr;
  sylv_handle* h = new sylv_handle();
  h->is_sub = true;
  h->opt = P->opt;
  h->s = SKK;
  h->lyap = false;
  h->mixed = P->mixed;
  h->stream = P->stream;
  h->own_stream = false;
  auto bail = [&](int rc) {
    std::string msg = g_err;
    sylv_destroy(h);
    g_err = msg;
    return rc;
  };
  if (cudaEventCreateWithFlags(&h->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev[1], cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(SYLV_ECUDA, "event"));
  if (cudaMallocHost(&h->st_host, 2 * sizeof(DevState)) != cudaSuccess) return bail(fail(SYLV_ECUDA, "pinned status"));
  int rc = alloc_fixed(h, &h->st, 1);
  if (rc) return bail(rc);
  const Side* src[2] = {&P->side[0], &P->side[P->lyap ? 0 : 1]};
  const int64_t n = P->side[0].n;
  const int64_t m = P->lyap ? n : P->side[1].n;
  double* rhs[2] = {(double*)P->sk[11].first, (double*)P->sk[12].first};  // Q (n x 8), Z (m x 8), row-major
  for (int i = 0; i < 2; ++i) {
    Side& sd = h->side[i];
    sd.n = src[i]->n;
    sd.nnz = src[i]->nnz;
    sd.rp = src[i]->rp;
    sd.ci = src[i]->ci;
    sd.vald = src[i]->vald;
    sd.valf = src[i]->valf;
    const int64_t rows = i == 0 ? n : m;
    if ((rc = alloc_fixed(h, &sd.C, rows * SKK))) return bail(rc);
    sylv::launch_unpack<double>(h->stream, rows, SKK, 1, rhs[i], rows * SKK, sd.C);
    if ((rc = alloc_fixed(h, &sd.RQR, 64)) || (rc = alloc_fixed(h, &sd.R1, 64)) || (rc = alloc_fixed(h, &sd.Rinv, 64)) ||
        (rc = alloc_fixed(h, (double**)&sd.RinvT, 64)))
      return bail(rc);
  }
  *out = h;
  return SYLV_OK;
}

void prof_add(sylv_handle* dst, const sylv_handle* src) {
  for (int i = 0; i < KC_NUM; ++i) {
    dst->prof.launches[i] += src->prof.launches[i];
    dst->prof.ms[i] += src->prof.ms[i];
    dst->prof.bytes[i] += src->prof.bytes[i];
    dst->prof.flops[i] += src->prof.flops[i];
  }
}

// Recurrence stop factor of a certified solve (sylv_options.stop_margin).
double stop_margin(const sylv_handle* h) { return h->opt.stop_margin > 0 ? h->opt.stop_margin : 0.4; }

// Outer driver: the factorized solve, then (unless disabled) the float64 true-residual
// certificate; SYLV_OK needs its bound <= tol.  In SYLV_FP64 the recurrence test of Algorithms
// 4.1/4.2 runs at stop_margin * tol, so that the bound holds at the first check; in SYLV_MIXED,
// refinement rounds A dX + dX B = (rank-8 part of R) until the bound meets tol.
template <typename T>
int run_solve(sylv_handle* h, int method, double tol, int maxit, sylv_info* info) {
  const double t0 = now_s();
  const int64_t launches0 = sylv::launch_counter();
  free_subs(h);
  h->true_rel = -1.0;
  h->true_bound = -1.0;
  h->refinements = 0;
  const bool check = !h->is_sub && (h->mixed || !h->opt.no_true_residual) && h->C1rm != nullptr;
  const double tol_in = (check && !h->mixed) ? tol * stop_margin(h) : tol;
  int rc = run_inner<T>(h, method, tol_in, maxit, info);
  h->total_iters = h->iters;
  h->total_width = h->width;
  if (check && (rc == SYLV_OK || rc == SYLV_ENOTCONV) && h->width > 0) {
    const int refine_max = h->opt.refine_max > 0 ? h->opt.refine_max : 12;
    const double tol_c = 0.05;  // a correction only has to beat the rank-8 truncation of R
    for (int round = 0;; ++round) {
      double est = 0.0, bound = 0.0;
      bool ok = false;
      cudaEvent_t pa = prof_begin(h);
      TRY(sketch<T>(h, &est, &bound, &ok));
      if (pa) {
        cudaEvent_t pb = prof_event(h);
        if (pb) {
          cudaEventRecord(pb, h->stream);
          cudaEventSynchronize(pb);
          float ms = 0.f;
          if (cudaEventElapsedTime(&ms, pa, pb) == cudaSuccess) {
            h->prof.launches[KC_RESID] += 1;
            h->prof.ms[KC_RESID] += ms;
          }
        }
      }
      h->prof.cur_k = -1;
      prof_finish(h, 1 << 30);
      h->true_rel = h->cnorm > 0 ? est / h->cnorm : 0.0;
      h->true_bound = h->cnorm > 0 ? bound / h->cnorm : 0.0;
      if (!h->mixed) {
        if (rc == SYLV_OK && h->true_bound > tol) {
          rc = SYLV_ENOTCONV;
          g_err = "the recurrence met its test but the float64 true residual is not certified below tol (bound " +
                  std::to_string(h->true_bound) + ", estimate " + std::to_string(h->true_rel) +
                  "); a smaller sylv_options.stop_margin runs further";
        }
        break;
      }
      if (h->true_bound <= tol) {
        rc = SYLV_OK;
        break;
      }
      rc = SYLV_ENOTCONV;
      if (!ok || round >= refine_max) break;
      sylv_handle* sub = nullptr;
      TRY(make_sub(h, &sub));
      h->subs.push_back(sub);
      sylv_info si;
      // a correction only has to reach tol_c (measured: 7-15 iterations); its basis is sized for
      // at most 40, so that a dozen rounds of a large workload fit in device memory beside the
      // main bases (an unconverged correction is still a correction)
      const int src = run_inner<T>(sub, method, tol_c, std::min(maxit, 40), &si);
      prof_add(h, sub);
      h->total_iters += sub->iters;
      h->total_width += sub->width;
      if (info)
        info->matvecs += (int64_t)(method == M_CG ? sub->iters : method == M_CR ? sub->iters + 1 : 2 * sub->iters);
      h->refinements += 1;
      if (src != SYLV_OK && src != SYLV_ENOTCONV) {
        rc = src;
        break;
      }
    }
  }
  h->status = rc;
  if (info) {
    info->status = rc;
    info->iters = (int32_t)h->total_iters;
    info->width = h->total_width;
    info->true_rel_res = h->true_rel;
    info->true_rel_bound = h->true_bound;
    info->refinements = h->refinements;
    info->solve_ms = (now_s() - t0) * 1e3;
    info->kernel_launches = sylv::launch_counter() - launches0;
  }
  return rc;
}


// ------------------------------------------------------------------ batched Lyapunov CG
int batch_items(sylv_handle* h, int chunk, std::vector<int2>& items, std::vector<sylv::BatchInst>& insts) {
  items.clear();
  for (size_t i = 0; i < h->batch.size(); ++i) {
    const int64_t n = h->batch[i]->side[0].n;
    insts[i].item_begin = (int)items.size();
    for (int64_t r0 = 0; r0 < n; r0 += chunk) items.push_back(make_int2((int)i, (int)r0));
    insts[i].item_end = (int)items.size();
  }
  if (items.size() > h->items_cap) {
    const size_t cap = items.size() * 2;
    if (h->d_items) cudaFree(h->d_items);
    if (h->b_gpart) cudaFree(h->b_gpart);
    if (h->b_spart) cudaFree(h->b_spart);
    h->d_items = nullptr;
    h->b_gpart = h->b_spart = nullptr;
    h->items_cap = 0;
    CU(cudaMalloc(&h->d_items, cap * sizeof(int2)));
    CU(cudaMalloc(&h->b_gpart, cap * 64 * sizeof(double)));
    CU(cudaMalloc(&h->b_spart, cap * 64 * sizeof(double)));
    h->items_cap = cap;
  }
  CU(cudaMemcpyAsync(h->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemcpyAsync(h->d_insts, insts.data(), insts.size() * sizeof(sylv::BatchInst), cudaMemcpyHostToDevice,
                     h->stream));
  CU(cudaStreamSynchronize(h->stream));  // the host vectors may change after return
  return SYLV_OK;
}

int batch_cg(sylv_handle* h, double tol, int maxit, sylv_info* info) {
  const double t0 = now_s();
  const double deadline = t0 + (h->opt.timeout_s > 0 ? h->opt.timeout_s : 3600.0);
  if (!(tol >= 0.0) || maxit < 0) return fail(SYLV_EINVAL, "tol must be >= 0 and maxit >= 0");
  const int count = (int)h->batch.size();
  cudaStream_t strm = h->stream;
  const int64_t launches0 = sylv::launch_counter();
  std::vector<sylv::BatchInst> insts(count);
  int maxs = 1;
  for (int i = 0; i < count; ++i) {
    sylv_handle* x = h->batch[i];
    TRY(ensure_capacity(x, M_CG, std::max(2, maxit + 1), maxit + 1));
    CU(cudaMemsetAsync(x->st, 0, sizeof(DevState), strm));
    const size_t l2 = (size_t)(x->lds * x->lds) * sizeof(double);
    for (double* p : {x->Xh, x->Rh, x->Ph, x->Qh, x->Th}) CU(cudaMemsetAsync(p, 0, l2, strm));
    CU(cudaMemsetAsync(x->side[0].H, 0, l2, strm));
    setup_qr<double>(x, 0);
    sylv::SmallCtx c = small_ctx(x);
    // certified instances stop their recurrence at stop_margin * tol (see run_solve)
    const double tol_in = h->opt.no_true_residual ? tol : tol * stop_margin(h);
    sylv::launch_init_small(strm, c, x->side[0].RQR, x->side[0].RQR, tol_in, 0);
    sylv::BatchInst& I = insts[i];
    std::memset(&I, 0, sizeof(I));
    I.n = x->side[0].n;
    I.s = (int)x->s;
    I.k = 0;
    I.rp = x->side[0].rp;
    I.ci = x->side[0].ci;
    I.val = x->side[0].vald;
    I.V = (double*)x->side[0].V;
    I.H = x->side[0].H;
    I.ldh = x->lds;
    I.X = x->Xh;
    I.R = x->Rh;
    I.P = x->Ph;
    I.Q = x->Qh;
    I.M = x->Th;
    I.lds = x->lds;
    I.st = x->st;
    I.hist = x->hist;
    I.R1 = x->side[0].R1;
    I.Rinv = x->side[0].Rinv;
    I.psm = x->psmall;
    maxs = std::max(maxs, I.s);
  }
  CU(cudaGetLastError());
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  sylv::BatchCtx bc{};
  bc.insts = h->d_insts;
  bc.count = count;
  bc.delta = deflate_tol(h);
  bc.running = h->d_running;
  bc.sgrid = 4 * sms;
  std::vector<int2> items;
  // autotuner: rows per work item x persistent grid size, timed on the batch itself
  // (sparse apply + Gram phases of the first iteration; the real iteration rewrites
  // everything they write)
  if (h->tuned_chunk == 0) {
    const int chunks[] = {512, 1024, 2048, 4096};
    const int mults[] = {1, 2, 4, 8};
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    const double tt0 = now_s();
    for (int ch : chunks)
      for (int mu : mults) {
        TRY(batch_items(h, ch, items, insts));
        bc.items = h->d_items;
        bc.nitems = (int)items.size();
        bc.chunk = ch;
        bc.grid = mu * sms;
        bc.gpart = h->b_gpart;
        bc.spart = h->b_spart;
        sylv::launch_batch_spmm_gram(strm, bc);
        CU(cudaEventRecord(e0, strm));
        for (int rep = 0; rep < 3; ++rep) sylv::launch_batch_spmm_gram(strm, bc);
        CU(cudaEventRecord(e1, strm));
        CU(cudaEventSynchronize(e1));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
          best = ms;
          h->tuned_chunk = ch;
          h->tuned_grid = mu * sms;
        }
      }
    h->tune_ms = (now_s() - tt0) * 1e3;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  TRY(batch_items(h, h->tuned_chunk, items, insts));
  bc.items = h->d_items;
  bc.nitems = (int)items.size();
  bc.chunk = h->tuned_chunk;
  bc.grid = h->tuned_grid;
  bc.gpart = h->b_gpart;
  bc.spart = h->b_spart;
  // one iteration of all instances as a CUDA graph (15 phase kernels)
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  CU(cudaStreamBeginCapture(strm, cudaStreamCaptureModeThreadLocal));
  const int64_t cap0 = sylv::launch_counter();
  sylv::launch_batch_iteration(strm, bc);
  const int64_t per_iteration = sylv::launch_counter() - cap0;  // captured, not launched
  sylv::launch_counter() = cap0;
  CU(cudaStreamEndCapture(strm, &g));
  cudaError_t ge = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (ge != cudaSuccess) return fail(SYLV_ECUDA, std::string("graph: ") + cudaGetErrorString(ge));
  const int poll = h->opt.poll_every > 0 ? h->opt.poll_every : 8;
  int slot = 0, pending = -1, k = 0;
  bool done = false;
  while (k < maxit && !done) {
    const int nrep = std::min(poll, maxit - k);
    for (int r = 0; r < nrep; ++r) CU(cudaGraphLaunch(h->graph, strm));
    sylv::launch_counter() += per_iteration * nrep;
    k += nrep;
    CU(cudaMemcpyAsync(&h->h_running[slot], h->d_running, sizeof(int), cudaMemcpyDeviceToHost, strm));
    CU(cudaEventRecord(h->ev[slot], strm));
    if (pending >= 0) {
      TRY(wait_status(h, pending, deadline));
      if (h->h_running[pending] == 0) done = true;
    }
    pending = slot;
    slot ^= 1;
  }
  CU(cudaStreamSynchronize(strm));
  // per-instance results, then the aggregate
  int agg = SYLV_OK;
  double worst = 0.0;
  int64_t width = 0, matvecs = 0;
  int maxk = 0;
  for (int i = 0; i < count; ++i) {
    sylv_handle* x = h->batch[i];
    DevState ds;
    CU(cudaMemcpy(&ds, x->st, sizeof(DevState), cudaMemcpyDeviceToHost));
    x->method = M_CG;
    x->iters = ds.iters;
    x->width = (int64_t)ds.iters * x->s;
    x->cert_valid = false;  // new bases
    x->cert_failed = false;
    x->total_iters = x->iters;
    x->total_width = x->width;
    x->nblocks = ds.iters + 1;
    int rc = ds.status == sylv::ST_CONVERGED ? SYLV_OK
             : ds.status == sylv::ST_RUNNING ? SYLV_ENOTCONV
             : ds.status == sylv::ST_BREAKDOWN ? SYLV_EBREAKDOWN
             : ds.status == sylv::ST_WAIT_TIMEOUT ? SYLV_ETIMEOUT : SYLV_ENONFINITE;
    x->status = rc;
    x->true_rel = -1.0;
    x->true_bound = -1.0;
    if (agg == SYLV_OK && rc != SYLV_OK) agg = rc;
    worst = std::max(worst, ds.r0 > 0 ? ds.rnorm / ds.r0 : 0.0);
    width += x->width;
    matvecs += ds.iters;
    maxk = std::max(maxk, ds.iters);
  }
  // float64 true residual of every instance (unless disabled), instances spread
  // over a pool of streams so the small ones run side by side
  double worst_true = -1.0, worst_bound = -1.0;
  if (!h->opt.no_true_residual) {
    if (h->pool.empty()) {
      h->pool.resize(16, nullptr);
      for (auto& ps : h->pool) CU(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
    }
    std::vector<sylv_handle*> todo;
    for (sylv_handle* x : h->batch)
      if (x->width > 0 && x->C1rm != nullptr) todo.push_back(x);
    for (size_t i = 0; i < todo.size(); ++i) {
      todo[i]->stream = h->pool[i % h->pool.size()];
      TRY(sketch_enqueue<double>(todo[i]));
    }
    int rc_all = SYLV_OK;
    for (sylv_handle* x : todo) {
      double est = 0.0, bound = 0.0;
      bool ok = false;
      const int rc = sketch_finish(x, &est, &bound, &ok);
      x->stream = h->stream;
      if (rc != SYLV_OK && rc_all == SYLV_OK) rc_all = rc;
      x->true_rel = x->cnorm > 0 ? est / x->cnorm : 0.0;
      x->true_bound = x->cnorm > 0 ? bound / x->cnorm : 0.0;
      worst_true = std::max(worst_true, x->true_rel);
      worst_bound = std::max(worst_bound, x->true_bound);
      // an instance whose recurrence converged is certified only if its bound meets tol
      if (x->status == SYLV_OK && x->true_bound > tol) {
        x->status = SYLV_ENOTCONV;
        if (agg == SYLV_OK) {
          agg = SYLV_ENOTCONV;
          g_err = "an instance's float64 true residual is not certified below tol (bound " +
                  std::to_string(x->true_bound) + ")";
        }
      }
    }
    if (rc_all != SYLV_OK) return rc_all;
  }
  h->method = M_CG;
  h->status = agg;
  h->iters = maxk;
  if (info) {
    info->status = agg;
    info->iters = maxk;
    info->matvecs = matvecs;
    info->width = width;
    info->rel_res = worst;
    info->true_rel_res = worst_true;
    info->true_rel_bound = worst_bound;
    info->solve_ms = (now_s() - t0) * 1e3;
    info->kernel_launches = sylv::launch_counter() - launches0;
  }
  return agg;
}

int solve(sylv_handle* h, int method, double tol, int32_t maxit, sylv_info* info) {
  if (!h) return fail(SYLV_EINVAL, "NULL handle");
  if (info) std::memset(info, 0, sizeof(*info));
  free_compressed(h);
  if (!h->batch.empty()) {
    if (method != M_CG) return fail(SYLV_EINVAL, "batched handles run factorized CG (Lyapunov) only");
    return batch_cg(h, tol, maxit, info);
  }
  return h->mixed ? run_solve<float>(h, method, tol, maxit, info) : run_solve<double>(h, method, tol, maxit, info);
}

template <typename T>
int unpack_to_host(sylv_handle* h, const Side& sd, int nb, double* out) {
  const int s = (int)h->s;
  const int64_t n = sd.n, bstride = n * s;
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)(256ll << 20) / (n * s * 8)));
  double* scratch = nullptr;
  CU(cudaMalloc(&scratch, (size_t)chunk * n * s * sizeof(double)));
  int rc = SYLV_OK;
  for (int b0 = 0; b0 < nb && rc == SYLV_OK; b0 += chunk) {
    const int cb = std::min(chunk, nb - b0);
    sylv::launch_unpack<T>(h->stream, n, s, cb, (const T*)sd.V + (int64_t)b0 * bstride, bstride, scratch);
    cudaError_t e = cudaMemcpyAsync(out + (int64_t)b0 * s * n, scratch, (size_t)cb * n * s * sizeof(double),
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = fail(SYLV_ECUDA, std::string("get_factors: ") + cudaGetErrorString(e));
  }
  cudaFree(scratch);
  return rc;
}

}  // namespace

namespace {
void free_subs(sylv_handle* h) {
  for (sylv_handle* sb : h->subs) sylv_destroy(sb);
  h->subs.clear();
}
}  // namespace

extern "C" {

void sylv_default_options(sylv_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = SYLV_FP64;
  opt->poll_every = 8;
  opt->refine_max = 12;
  opt->timeout_s = 3600.0;
}

int sylv_create(const sylv_csr* A, const sylv_csr* B, const double* C1, const double* C2, int64_t s,
                const sylv_options* opt, sylv_handle** out) {
  g_err.clear();
  if (!out) return fail(SYLV_EINVAL, "out is NULL");
  *out = nullptr;
  sylv_options o;
  sylv_default_options(&o);
  if (opt) o = *opt;
  if (s < 1 || s > 8) return fail(SYLV_EINVAL, "s must be in [1, 8]");
  if (o.precision != SYLV_FP64 && o.precision != SYLV_MIXED) return fail(SYLV_EINVAL, "unknown precision");
  if (o.basis_gemm < 0 || o.basis_gemm > 2) return fail(SYLV_EINVAL, "basis_gemm must be 0, 1 or 2");
  if (o.cert_gemm < 0 || o.cert_gemm > 2) return fail(SYLV_EINVAL, "cert_gemm must be 0, 1 or 2");
  TRY(check_csr(A, "A", -1));
  const bool lyap = o.lyapunov != 0;
  if (lyap) {
    if (B != nullptr || C2 != nullptr) return fail(SYLV_EINVAL, "Lyapunov case: pass B = NULL and C2 = NULL");
  } else {
    TRY(check_csr(B, "B", -1));
    if (!C2) return fail(SYLV_EINVAL, "C2 is NULL");
  }
  if (!C1) return fail(SYLV_EINVAL, "C1 is NULL");
  if (A->nrows < s || (!lyap && B->nrows < s)) return fail(SYLV_EINVAL, "need n, m >= s");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(SYLV_ECUDA, "no CUDA device");
  }
  sylv_handle* h = new sylv_handle();
  h->opt = o;
  h->s = s;
  h->lyap = lyap;
  h->mixed = o.precision == SYLV_MIXED;
  auto bail = [&](int rc) {
    std::string msg = g_err;
    sylv_destroy(h);
    g_err = msg;
    return rc;
  };
  if (o.cuda_stream) {
    h->stream = (cudaStream_t)o.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(fail(SYLV_ECUDA, "stream"));
    h->own_stream = true;
  }
  if (cudaEventCreateWithFlags(&h->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev[1], cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(SYLV_ECUDA, "event"));
  if (cudaMallocHost(&h->st_host, 2 * sizeof(DevState)) != cudaSuccess) return bail(fail(SYLV_ECUDA, "pinned status"));
  int rc = alloc_fixed(h, &h->st, 1);
  if (rc) return bail(rc);
  rc = upload_operator(h, h->side[0], A, false);
  if (!rc) rc = upload_rhs(h, h->side[0], C1);
  if (!rc && !lyap) rc = upload_operator(h, h->side[1], B, true);
  if (!rc && !lyap) rc = upload_rhs(h, h->side[1], C2);
  if (!rc && (h->mixed || !o.no_true_residual)) rc = prepare_residual_ops(h, A, B);
  if (rc) return bail(rc);
  *out = h;
  return SYLV_OK;
}

int sylv_cg(sylv_handle* h, double tol, int32_t maxit, sylv_info* info) {
  g_err.clear();
  return solve(h, M_CG, tol, maxit, info);
}

int sylv_bicgstab(sylv_handle* h, double tol, int32_t maxit, sylv_info* info) {
  g_err.clear();
  return solve(h, M_BICG, tol, maxit, info);
}

int sylv_cgs(sylv_handle* h, double tol, int32_t maxit, sylv_info* info) {
  g_err.clear();
  return solve(h, M_CGS, tol, maxit, info);
}

int sylv_cr(sylv_handle* h, double tol, int32_t maxit, sylv_info* info) {
  g_err.clear();
  return solve(h, M_CR, tol, maxit, info);
}

int sylv_gpbicg(sylv_handle* h, double tol, int32_t maxit, sylv_info* info) {
  g_err.clear();
  return solve(h, M_GPBICG, tol, maxit, info);
}

int sylv_create_batch(int32_t count, const sylv_csr* A, const sylv_csr* B, const double* const* C1,
                      const double* const* C2, const int64_t* s, const sylv_options* opt, sylv_handle** out) {
  g_err.clear();
  if (!out) return fail(SYLV_EINVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || !A || !C1 || !s) return fail(SYLV_EINVAL, "need count >= 1 and A, C1, s arrays");
  sylv_options o;
  sylv_default_options(&o);
  if (opt) o = *opt;
  if (!o.lyapunov || B != nullptr || C2 != nullptr)
    return fail(SYLV_EINVAL, "batched mode solves Lyapunov equations: set lyapunov = 1, B = C2 = NULL");
  if (o.precision != SYLV_FP64) return fail(SYLV_EINVAL, "batched mode runs in SYLV_FP64");
  sylv_handle* h = new sylv_handle();
  h->opt = o;
  h->lyap = true;
  h->s = 0;
  auto bail = [&](int rc) {
    std::string msg = g_err;
    sylv_destroy(h);
    g_err = msg;
    return rc;
  };
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    delete h;
    return fail(SYLV_ECUDA, "no CUDA device");
  }
  if (o.cuda_stream) {
    h->stream = (cudaStream_t)o.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(fail(SYLV_ECUDA, "stream"));
    h->own_stream = true;
  }
  if (cudaEventCreateWithFlags(&h->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev[1], cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(SYLV_ECUDA, "event"));
  if (cudaMallocHost(&h->h_running, 2 * sizeof(int)) != cudaSuccess) return bail(fail(SYLV_ECUDA, "pinned"));
  int rc = alloc_fixed(h, &h->d_running, 1);
  if (!rc) rc = alloc_fixed(h, &h->d_insts, (size_t)count);
  if (rc) return bail(rc);
  sylv_options io = o;
  io.cuda_stream = h->stream;
  io.profile = 0;
  for (int i = 0; i < count; ++i) {
    sylv_handle* x = nullptr;
    rc = sylv_create(&A[i], nullptr, C1[i], nullptr, s[i], &io, &x);
    if (rc) {
      g_err = "instance " + std::to_string(i) + ": " + g_err;
      return bail(rc);
    }
    h->batch.push_back(x);
  }
  *out = h;
  return SYLV_OK;
}

int sylv_batch_instance(sylv_handle* h, int32_t inst, sylv_handle** out) {
  if (!h || !out) return fail(SYLV_EINVAL, "NULL argument");
  *out = nullptr;
  if (h->batch.empty()) return fail(SYLV_EINVAL, "not a batched handle");
  if (inst < 0 || inst >= (int32_t)h->batch.size()) return fail(SYLV_EINVAL, "instance index out of range");
  *out = h->batch[inst];
  return SYLV_OK;
}

int sylv_get_factors(sylv_handle* h, double* V, double* Xhat, double* W, int64_t* r) {
  if (!h) return fail(SYLV_EINVAL, "NULL handle");
  if (!h->batch.empty()) return fail(SYLV_EINVAL, "batched handle: use sylv_batch_instance");
  if (h->method == M_NONE) return fail(SYLV_ESTATE, "no solve yet");
  if (h->comp_q >= 0) {  // compressed: V_q, diag(s_q), W_q
    const int64_t q = h->comp_q;
    if (r) *r = q;
    if (q == 0) return SYLV_OK;
    const int64_t n = h->side[0].n, m = h->side[h->lyap ? 0 : 1].n;
    if (Xhat) {
      std::memset(Xhat, 0, (size_t)q * q * sizeof(double));
      for (int64_t i = 0; i < q; ++i) Xhat[i + i * q] = h->comp_s[i];
    }
    if (V) CU(cudaMemcpy(V, h->comp_V, (size_t)n * q * sizeof(double), cudaMemcpyDeviceToHost));
    if (W) CU(cudaMemcpy(W, h->comp_W, (size_t)m * q * sizeof(double), cudaMemcpyDeviceToHost));
    return SYLV_OK;
  }
  const int64_t R = h->total_width;
  if (r) *r = R;
  if (R == 0) return SYLV_OK;
  std::vector<sylv_handle*> rounds{h};
  for (sylv_handle* sb : h->subs) rounds.push_back(sb);
  if (Xhat) std::memset(Xhat, 0, (size_t)R * R * sizeof(double));  // block diagonal over the rounds
  int64_t off = 0;
  for (sylv_handle* x : rounds) {
    const int64_t w = x->width;
    if (w == 0) continue;
    const int nb = (int)(w / x->s);
    if (Xhat) {
      CU(cudaMemcpy2DAsync(Xhat + off + off * R, R * sizeof(double), x->Xh, x->lds * sizeof(double),
                           w * sizeof(double), w, cudaMemcpyDeviceToHost, x->stream));
      CU(cudaStreamSynchronize(x->stream));
    }
    for (int i = 0; i < 2; ++i) {
      double* dst = i == 0 ? V : W;
      if (!dst) continue;
      const Side& sd = x->side[(i == 1 && !x->lyap) ? 1 : 0];
      double* at = dst + off * sd.n;
      TRY(x->mixed ? unpack_to_host<float>(x, sd, nb, at) : unpack_to_host<double>(x, sd, nb, at));
    }
    off += w;
  }
  return SYLV_OK;
}

constexpr int kJacobiSweeps = 100;  // sweep limit of the compression's Jacobi SVD

int sylv_compress(sylv_handle* h, double tol, int64_t* q_out) {
  if (!h) return fail(SYLV_EINVAL, "NULL handle");
  if (!h->batch.empty()) return fail(SYLV_EINVAL, "batched handle: compression needs a single solve");
  if (h->method == M_NONE) return fail(SYLV_ESTATE, "no solve yet");
  if (!(tol >= 0.0)) return fail(SYLV_EINVAL, "tol must be >= 0");
  if (h->mixed || !arnoldi_method(h->method) || !h->subs.empty())
    return fail(SYLV_EINVAL, "compression needs the orthonormal float64 bases of BiCGSTAB, CGS or GPBiCG");
  if (h->comp_q >= 0) return fail(SYLV_ESTATE, "already compressed");
  const int r = (int)h->width;
  cudaStream_t strm = h->stream;
  std::vector<void*> tmp;
  auto cleanup = [&]() {
    for (void* p : tmp) cudaFree(p);
  };
  auto dalloc = [&](void** p, size_t bytes) -> int {
    if (cudaMalloc(p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
      cudaGetLastError();
      return fail(SYLV_ENOMEM, "compression buffers");
    }
    tmp.push_back(*p);
    return SYLV_OK;
  };
  int rc = SYLV_OK;
  double *G = nullptr, *Z = nullptr, *sig = nullptr, *scale = nullptr;
  int *pairs = nullptr, *rotated = nullptr, *cols = nullptr;
  const size_t rr = (size_t)std::max(r, 1) * std::max(r, 1);
  std::vector<int> sched;
  sylv::jacobi_schedule(r, sched);
  if ((rc = dalloc((void**)&G, rr * 8)) || (rc = dalloc((void**)&Z, rr * 8)) || (rc = dalloc((void**)&sig, r * 8 + 8)) ||
      (rc = dalloc((void**)&scale, r * 8 + 8)) || (rc = dalloc((void**)&cols, r * 4 + 4)) ||
      (rc = dalloc((void**)&rotated, 4)) || (rc = dalloc((void**)&pairs, sched.size() * 4 + 4))) {
    cleanup();
    return rc;
  }
  auto run = [&]() -> int {
    if (r > 0) {
      CU(cudaMemcpy2DAsync(G, (size_t)r * 8, h->Xh, (size_t)h->lds * 8, (size_t)r * 8, r, cudaMemcpyDeviceToDevice,
                           strm));
      std::vector<double> eye((size_t)r * r, 0.0);
      for (int i = 0; i < r; ++i) eye[(size_t)i * r + i] = 1.0;
      CU(cudaMemcpyAsync(Z, eye.data(), rr * 8, cudaMemcpyHostToDevice, strm));
      CU(cudaMemcpyAsync(pairs, sched.data(), sched.size() * 4, cudaMemcpyHostToDevice, strm));
      const int r2 = r + (r & 1);
      // ||X^||_F for the rounding floor of the column norms
      sylv::launch_column_norms(strm, r, G, r, sig);
      std::vector<double> c0(r);
      CU(cudaMemcpyAsync(c0.data(), sig, (size_t)r * 8, cudaMemcpyDeviceToHost, strm));
      CU(cudaStreamSynchronize(strm));
      double fro2 = 0.0;
      for (double v : c0) fro2 += v * v;
      const double floor_ = (double)r * 2.220446049250313e-16 * std::sqrt(fro2), tau = floor_ * floor_;
      int sweeps = 0;
      for (; sweeps < kJacobiSweeps; ++sweeps) {  // one-sided Jacobi: sweep until no pair rotates
        CU(cudaMemsetAsync(rotated, 0, 4, strm));
        for (int round = 0; round < r2 - 1; ++round)
          sylv::launch_jacobi_round(strm, r, G, Z, r, pairs + (size_t)round * r2, 1e-14, tau, rotated);
        int hrot = 0;
        CU(cudaMemcpyAsync(&hrot, rotated, 4, cudaMemcpyDeviceToHost, strm));
        CU(cudaStreamSynchronize(strm));
        if (hrot == 0) break;
      }
      if (sweeps == kJacobiSweeps) return fail(SYLV_ENOTCONV, "Jacobi SVD did not converge");
      sylv::launch_column_norms(strm, r, G, r, sig);
    }
    std::vector<double> s(r);
    if (r > 0) CU(cudaMemcpyAsync(s.data(), sig, (size_t)r * 8, cudaMemcpyDeviceToHost, strm));
    CU(cudaStreamSynchronize(strm));
    std::vector<int> perm(r);
    for (int i = 0; i < r; ++i) perm[i] = i;
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return s[a] > s[b]; });
    // q: the smallest rank whose discarded singular values have norm <= tol * ||s||
    std::vector<double> tail(r + 1, 0.0);
    for (int i = r - 1; i >= 0; --i) tail[i] = tail[i + 1] + s[perm[i]] * s[perm[i]];
    const double total = tail[0];  // the same sum, so tol >= 1 gives q = 0
    int q = r;
    for (int k = 0; k <= r; ++k)
      if (std::sqrt(tail[k]) <= tol * std::sqrt(total)) {
        q = k;
        break;
      }
    std::vector<double> inv(q), ones(q, 1.0);
    h->comp_s.resize(q);
    for (int k = 0; k < q; ++k) {
      h->comp_s[k] = s[perm[k]];
      inv[k] = s[perm[k]] > 0.0 ? 1.0 / s[perm[k]] : 0.0;
    }
    const Side& sa = h->side[0];
    const Side& sb = h->side[h->lyap ? 0 : 1];
    if (cudaMalloc(&h->comp_V, std::max<size_t>((size_t)sa.n * q * 8, 256)) != cudaSuccess ||
        cudaMalloc(&h->comp_W, std::max<size_t>((size_t)sb.n * q * 8, 256)) != cudaSuccess) {
      cudaGetLastError();
      return fail(SYLV_ENOMEM, "compressed factors");
    }
    if (q > 0) {
      CU(cudaMemcpyAsync(cols, perm.data(), (size_t)q * 4, cudaMemcpyHostToDevice, strm));
      CU(cudaMemcpyAsync(scale, inv.data(), (size_t)q * 8, cudaMemcpyHostToDevice, strm));
      sylv::launch_apply_blocks(strm, sa.n, (int)h->s, r, (const double*)sa.V, sa.n * h->s, G, r, cols, scale, q,
                                h->comp_V);  // V U_q, U_q = G(:, kept) / s
      CU(cudaMemcpyAsync(scale, ones.data(), (size_t)q * 8, cudaMemcpyHostToDevice, strm));
      sylv::launch_apply_blocks(strm, sb.n, (int)h->s, r, (const double*)sb.V, sb.n * h->s, Z, r, cols, scale, q,
                                h->comp_W);  // W Z_q
      CU(cudaGetLastError());
      CU(cudaStreamSynchronize(strm));
    }
    h->comp_q = q;
    if (q_out) *q_out = q;
    return SYLV_OK;
  };
  rc = run();
  cleanup();
  if (rc != SYLV_OK && h->comp_q < 0) {
    if (h->comp_V) cudaFree(h->comp_V);
    if (h->comp_W) cudaFree(h->comp_W);
    h->comp_V = h->comp_W = nullptr;
  }
  return rc;
}

int sylv_get_history(sylv_handle* h, double* hist, int64_t cap, int64_t* len) {
  if (!h) return fail(SYLV_EINVAL, "NULL handle");
  if (h->method == M_NONE) return fail(SYLV_ESTATE, "no solve yet");
  const int64_t L = h->iters + 1;
  if (len) *len = L;
  if (hist && cap > 0) {
    CU(cudaMemcpyAsync(hist, h->hist, std::min(cap, L) * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  return SYLV_OK;
}

int sylv_get_hessenberg(sylv_handle* h, int32_t side, double* H, int64_t cap, int32_t* nblocks) {
  if (!h) return fail(SYLV_EINVAL, "NULL handle");
  if (h->method == M_NONE) return fail(SYLV_ESTATE, "no solve yet");
  if (side < 0 || side > 1) return fail(SYLV_EINVAL, "side must be 0 or 1");
  const int nb = h->nblocks;
  if (nblocks) *nblocks = nb;
  if (!H) return SYLV_OK;
  const int64_t rows = (int64_t)nb * h->s, cols = (int64_t)(nb - 1) * h->s;
  if (cap < rows * cols) return fail(SYLV_EINVAL, "H buffer too small");
  const Side& sd = h->side[(side == 1 && !h->lyap) ? 1 : 0];
  if (rows > 0 && cols > 0) {
    CU(cudaMemcpy2DAsync(H, rows * sizeof(double), sd.H, h->lds * sizeof(double), rows * sizeof(double), cols,
                         cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  return SYLV_OK;
}

int sylv_small_operator(sylv_handle* h, int64_t r, const double* Z, double* out) {
  if (!h) return fail(SYLV_EINVAL, "NULL handle");
  if (!h->batch.empty()) return fail(SYLV_EINVAL, "not available on a batched handle");
  if (h->method == M_NONE || h->Qh == nullptr) return fail(SYLV_ESTATE, "no solve yet");
  const int64_t s = h->s, rp = r + s;
  // H_{k+1,k} and G_{k+1,k} must be built: r columns and r + s rows of the last solve's bases
  if (r < 1 || r % s != 0 || r > (int64_t)(h->nblocks - 1) * s || rp > h->lds || !Z || !out)
    return fail(SYLV_EINVAL, "r must be a positive multiple of s within the last solve's basis width");
  DevState* st = nullptr;
  CU(cudaMalloc(&st, sizeof(DevState)));  // a status word of its own: the solve's may say "stopped"
  int rc = SYLV_OK;
  const size_t ld = (size_t)h->lds * sizeof(double);
  sylv::SmallCtx c = small_ctx(h);
  c.st = st;
  cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevState), h->stream);
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(h->Ph, ld, Z, r * sizeof(double), r * sizeof(double), r,
                                              cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Qh, 0, (size_t)h->lds * rp * sizeof(double), h->stream);
  if (e == cudaSuccess) {
    sylv::launch_sylv_gemm(h->stream, c, (int)r, h->Ph, h->Qh, false);
    e = cudaGetLastError();
  }
  DevState ds{};
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(out, rp * sizeof(double), h->Qh, ld, rp * sizeof(double), rp,
                                              cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ds, st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) rc = fail(SYLV_ECUDA, std::string("sylv_small_operator: ") + cudaGetErrorString(e));
  else if (ds.status == sylv::ST_WAIT_TIMEOUT) rc = fail(SYLV_ETIMEOUT, "a device-side wait gave up");
  else if (ds.status != sylv::ST_RUNNING) rc = fail(SYLV_ENONFINITE, "non-finite value in the small operator");
  cudaFree(st);
  return rc;
}

int sylv_set_timeout(sylv_handle* h, double timeout_s) {
  if (!h) return fail(SYLV_EINVAL, "NULL handle");
  if (!(timeout_s >= 0.0)) return fail(SYLV_EINVAL, "timeout_s must be >= 0");
  h->opt.timeout_s = timeout_s;
  for (sylv_handle* b : h->batch) b->opt.timeout_s = timeout_s;
  return SYLV_OK;
}

int sylv_apply(sylv_handle* h, int32_t side, const double* X, double* Y, int64_t k) {
  if (!h) return fail(SYLV_EINVAL, "NULL handle");
  if (side < 0 || side > 1 || k < 1 || k > 8 || !X || !Y) return fail(SYLV_EINVAL, "bad sylv_apply arguments");
  const Side& sd = h->side[(side == 1 && !h->lyap) ? 1 : 0];
  const int64_t n = sd.n;
  const size_t fsz = h->mixed ? sizeof(float) : sizeof(double);
  double* xc = nullptr;
  void *xb = nullptr, *yb = nullptr;
  CU(cudaMalloc(&xc, n * k * sizeof(double)));
  int rc = SYLV_OK;
  cudaError_t e = cudaMalloc(&xb, n * k * fsz);
  if (e == cudaSuccess) e = cudaMalloc(&yb, n * k * fsz);
  if (e == cudaSuccess) e = cudaMemcpyAsync(xc, X, n * k * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    if (h->mixed) {
      sylv::launch_pack<float>(h->stream, n, (int)k, xc, (float*)xb);
      sylv::launch_spmm<float>(h->stream, nullptr, n, (int)k, sd.rp, sd.ci, sd.valf, (float*)xb, (float*)yb, nullptr,
                               nullptr, 0);
      sylv::launch_unpack<float>(h->stream, n, (int)k, 1, (float*)yb, n * k, xc);
    } else {
      sylv::launch_pack<double>(h->stream, n, (int)k, xc, (double*)xb);
      sylv::launch_spmm<double>(h->stream, nullptr, n, (int)k, sd.rp, sd.ci, sd.vald, (double*)xb, (double*)yb,
                                nullptr, nullptr, 0);
      sylv::launch_unpack<double>(h->stream, n, (int)k, 1, (double*)yb, n * k, xc);
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(Y, xc, n * k * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) rc = fail(e == cudaErrorMemoryAllocation ? SYLV_ENOMEM : SYLV_ECUDA, cudaGetErrorString(e));
  cudaFree(xc);
  cudaFree(xb);
  cudaFree(yb);
  return rc;
}

int sylv_get_profile(sylv_handle* h, sylv_kernel_stat* out, int32_t cap, int32_t* count) {
  if (!h) return fail(SYLV_EINVAL, "NULL handle");
  int cnt = 0;
  if (h->prof.valid) {
    for (int i = 0; i < KC_NUM; ++i) {
      if (h->prof.launches[i] == 0) continue;
      if (out && cnt < cap) {
        sylv_kernel_stat& e = out[cnt];
        std::memset(&e, 0, sizeof(e));
        std::strncpy(e.name, kKcNames[i], sizeof(e.name) - 1);
        e.launches = h->prof.launches[i];
        e.ms = h->prof.ms[i];
        e.bytes = h->prof.bytes[i];
        e.flops = h->prof.flops[i];
      }
      ++cnt;
    }
  }
  if (count) *count = cnt;
  return SYLV_OK;
}

const char* sylv_strerror(int status) {
  switch (status) {
    case SYLV_OK: return "converged";
    case SYLV_EINVAL: return "invalid argument";
    case SYLV_ENOMEM: return "out of device memory";
    case SYLV_ENOTCONV: return "maximum number of iterations reached";
    case SYLV_EBREAKDOWN: return "breakdown (zero denominator or rank-deficient block)";
    case SYLV_ENONFINITE: return "non-finite value";
    case SYLV_ETIMEOUT: return "timed out waiting for the device";
    case SYLV_ECUDA: return "CUDA error";
    case SYLV_ESTATE: return "call out of order";
    default: return "unknown status";
  }
}

const char* sylv_last_error(void) { return g_err.c_str(); }

void sylv_destroy(sylv_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (sylv_handle* x : h->batch) sylv_destroy(x);
  h->batch.clear();
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->h_running) cudaFreeHost(h->h_running);
  for (auto& ps : h->pool)
    if (ps) cudaStreamDestroy(ps);
  if (h->sk_host) cudaFreeHost(h->sk_host);
  free_subs(h);
  free_sketch(h);
  free_compressed(h);
  free_solve(h);
  if (h->cert_mem) cudaFree(h->cert_mem);
  for (void* p : h->fixed_allocs) cudaFree(p);
  h->fixed_allocs.clear();
  if (h->st_host) cudaFreeHost(h->st_host);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : h->prof.pool) cudaEventDestroy(e);
  for (auto& sb : h->sbas)
    if (sb) cudaStreamDestroy(sb);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  for (auto& pr : h->ev_bas)
    for (auto& e : pr)
      if (e) cudaEventDestroy(e);
  for (auto& e : h->ev_small)
    if (e) cudaEventDestroy(e);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // extern "C"
