// Internal declarations of libpint (GB300 / sm_103a). Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>
#include <utility>
#include <string>
#include <vector>

#include "pint.h"

#include <nvtx3/nvToolsExt.h>

namespace pint {

constexpr int kSellC = 32;          // SELL slice height = warp size
// Layout of pint_ctx_s::d_small (doubles)
constexpr int kSmallNormPartial = 0;      // 512 x 16 column-norm partials
constexpr int kSmallChol = 8192;          // CholQR scratch (4 x 256)
constexpr int kSmallScratch = 10240;      // small per-call vectors
constexpr int kSmallDoubles = 16384;
constexpr int kMaxS = PINT_MAX_S;

// ----------------------------------------------------------------- errors
struct Error {
  int code;
  std::string msg;
};

#define PINT_CUDA(call)                                                      \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      throw ::pint::Error{PINT_ERR_CUDA, std::string(#call) + ": " +         \
                                             cudaGetErrorString(e_)};        \
  } while (0)

#define PINT_REQUIRE(cond, code, text)                                       \
  do {                                                                       \
    if (!(cond)) throw ::pint::Error{(code), (text)};                        \
  } while (0)

inline void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    throw Error{PINT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

// ------------------------------------------------- checked builds
// With -DPINT_BOUNDS (build.build(bounds=True) makes libpint_bounds.so) an
// index gathered from a matrix (a CSR or SELL column) is checked against its
// bound before use. A bad one is counted and the first is recorded as (site,
// index, bound) in this translation unit's record, and the access is
// skipped. Without the flag the check is the constant true and compiles
// away. Sites: 1 coupled residual, 2 SELL SpMM, 3 batched operator rows,
// 99 the test entry pint_test_bounds.
#ifdef PINT_BOUNDS
static __device__ unsigned long long g_pint_bounds[4];   // count, site, index, bound
__device__ __forceinline__ bool pint_index_ok(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  if (atomicAdd(&g_pint_bounds[0], 1ULL) == 0ULL) {
    g_pint_bounds[1] = (unsigned long long)site;
    g_pint_bounds[2] = (unsigned long long)i;
    g_pint_bounds[3] = (unsigned long long)n;
  }
  return false;
}
#define PINT_INDEX_OK(i, n, site) ::pint::pint_index_ok((long long)(i), (long long)(n), (site))
// this translation unit's record (count, site, index, bound), then cleared
static inline void pint_bounds_take(unsigned long long* out) {
  cudaMemcpyFromSymbol(out, g_pint_bounds, 4 * sizeof(unsigned long long));
  const unsigned long long z[4] = {0, 0, 0, 0};
  cudaMemcpyToSymbol(g_pint_bounds, z, sizeof(z));
}
#else
#define PINT_INDEX_OK(i, n, site) true
static inline void pint_bounds_take(unsigned long long* out) {
  out[0] = out[1] = out[2] = out[3] = 0;
}
#endif
void bounds_take_spmm(unsigned long long* out);    // spmm.cu
void bounds_take_batch(unsigned long long* out);   // batch.cu

// -------------------------------------------------------- device helpers
template <typename T>
struct AccOf { using type = T; };
template <>
struct AccOf<__nv_bfloat16> { using type = float; };

__device__ __forceinline__ double to_acc(double v, double) { return v; }
__device__ __forceinline__ float to_acc(float v, float) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v, float) { return __bfloat162float(v); }

// Load the s values of one block-vector row into registers. EXACT: s == S and
// 16-byte vector loads where the row is a multiple of 16 bytes; otherwise
// scalar loads guarded by k < s (zero-filled).
template <int S, bool EXACT>
__device__ __forceinline__ void load_row(const double* __restrict__ p, int s, double (&x)[S]) {
  if constexpr (EXACT && S % 2 == 0) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int i = 0; i < S / 2; ++i) {
      double2 v = __ldg(q + i);
      x[2 * i] = v.x;
      x[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < S; ++k) x[k] = (EXACT || k < s) ? __ldg(p + k) : 0.0;
  }
}

template <int S, bool EXACT>
__device__ __forceinline__ void load_row(const float* __restrict__ p, int s, float (&x)[S]) {
  if constexpr (EXACT && S % 4 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < S / 4; ++i) {
      float4 v = __ldg(q + i);
      x[4 * i] = v.x; x[4 * i + 1] = v.y; x[4 * i + 2] = v.z; x[4 * i + 3] = v.w;
    }
  } else if constexpr (EXACT && S == 2) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    x[0] = v.x; x[1] = v.y;
  } else {
#pragma unroll
    for (int k = 0; k < S; ++k) x[k] = (EXACT || k < s) ? __ldg(p + k) : 0.0f;
  }
}

// Same as load_row but for data written earlier in the same launch by other
// CTAs: bypasses L1 (ld.global.cg).
template <int S, bool EXACT, typename T>
__device__ __forceinline__ void load_row_cg(const T* p, int s, T (&x)[S]) {
#pragma unroll
  for (int k = 0; k < S; ++k) x[k] = (EXACT || k < s) ? __ldcg(p + k) : T(0);
}

template <int S, bool EXACT>
__device__ __forceinline__ void store_row(double* __restrict__ p, int s, const double (&x)[S]) {
  if constexpr (EXACT && S % 2 == 0) {
    double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int i = 0; i < S / 2; ++i) q[i] = make_double2(x[2 * i], x[2 * i + 1]);
  } else {
#pragma unroll
    for (int k = 0; k < S; ++k)
      if (EXACT || k < s) p[k] = x[k];
  }
}

template <int S, bool EXACT>
__device__ __forceinline__ void store_row(float* __restrict__ p, int s, const float (&x)[S]) {
  if constexpr (EXACT && S % 4 == 0) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int i = 0; i < S / 4; ++i)
      q[i] = make_float4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
  } else if constexpr (EXACT && S == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
  } else {
#pragma unroll
    for (int k = 0; k < S; ++k)
      if (EXACT || k < s) p[k] = x[k];
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// s x s coupling matrices passed by value (kernel parameter space).
struct Coupling {
  double A1[kMaxS * kMaxS];
  double A2[kMaxS * kMaxS];
};

// ---------------------------------------------------------- SELL-32 format
// Rows in natural order (sigma = 1), slice q = rows [32q, 32q+32). Element
// (row 32q+l, slot t) at slice_ptr[q] + 32 t + l. Padding entries carry the
// row itself as column and value 0.
struct SellPattern {
  int64_t n = 0, nslices = 0, nelem = 0;
  int64_t* slice_ptr = nullptr;   // device, nslices + 1
  int* col = nullptr;             // device, nelem
  int64_t* csr_to_sell = nullptr; // device, nnz: SELL position of CSR entry
};

}  // namespace pint

namespace pint {
// Kernel families for the optional CUDA-event profiler (pint_profile_*).
enum ProfFamily {
  PF_COUPLED = 0,  // fused coupled residual (k_coupled, k_nl_residual)
  PF_SPMM,         // inner operator apply (k_spmm)
  PF_GRAM,         // block Gram products (k_gram + reduce)
  PF_UPDATE,       // block AXPY with a small matrix (k_update)
  PF_CHOLQR,       // CholQR pieces (k_chol, k_rowmul, small mm)
  PF_HESS,         // Hessenberg least squares (k_hess_step, k_backsolve, init)
  PF_ILU,          // ILU(0) factor and sweeps
  PF_NORM,         // column norms
  PF_VEC,          // outer update, casts, axpy, shift, B0 terms
  PF_NL,           // nonlinear pointwise / Jacobian / eval kernels
  PF_COUNT
};
struct ProfRec {
  int fam;
  cudaEvent_t a, b;
  double bytes, flops;
};
}  // namespace pint

// ------------------------------------------------------------ opaque types
struct pint_ctx_s {
  int device = 0;
  int num_sms = 0;
  size_t budget = 0;
  size_t used = 0;
  std::string err;
  // pinned host words for convergence flags and small reductions
  int* h_flag = nullptr;
  double* h_small = nullptr;     // 4096 doubles
  // scratch for reductions (Gram partials, norms)
  double* d_partial = nullptr;
  size_t partial_bytes = 0;
  double* d_small = nullptr;     // 65536 doubles of small dense state
  int* d_flag = nullptr;         // 64 ints
  long launches = 0;
  // profiler
  bool prof_on = false;
  bool nvtx_on = false;          // an NVTX range per kernel family launch
  bool gram_fuse = true;         // block CGS2: first update fused into the second Gram
  // relative residual ||R_k|| / ||F_k|| of every column at every outer (or
  // Newton) iteration since the last reset: rows of hist_s values
  std::vector<double> hist;
  int hist_s = 0;
  std::vector<pint::ProfRec> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[pint::PF_COUNT] = {};
  double prof_bytes[pint::PF_COUNT] = {};
  double prof_flops[pint::PF_COUNT] = {};
  long prof_launches[pint::PF_COUNT] = {};
};

namespace pint {
struct IluState;     // ilu.cu
struct KrylovWork;   // krylov.cu
}  // namespace pint

struct pint_op_s {
  pint_ctx ctx = nullptr;
  int64_t n = 0, nnz = 0;
  // CSR of K (device) and host pattern copy
  int* rowptr = nullptr;
  int* colind = nullptr;
  double* Kval = nullptr;
  double* Mdiag = nullptr;       // nullptr -> M = I
  int* diagpos = nullptr;        // device, CSR position of the diagonal
  std::vector<int> h_rowptr, h_colind;
  pint::SellPattern sell;
  // structured-grid shape when the pattern is the natural-order 5/7-point
  // stencil built by the FV constructors (0 otherwise)
  int grid_nx = 0, grid_ny = 0, grid_nz = 0;
  double* sellK = nullptr;       // K values in SELL (float64)
  // coupling
  int s = 0;
  double A1[pint::kMaxS * pint::kMaxS] = {};
  double A2[pint::kMaxS * pint::kMaxS] = {};
  double alpha = 0.0, beta = 0.0;
  // inner operator J = alpha M + beta K (valid while j_valid)
  bool j_valid = false;
  double* Jval = nullptr;        // CSR float64
  double* Jdiag = nullptr;       // diag(J)
  double* Jinvdiag = nullptr;    // 1 / diag(J)
  // SELL copies of J: [precision][jacobi_scaled]
  void* sellJ[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
  // stencil copies of J (grid operators only): [precision][jacobi_scaled],
  // 8 coefficients per row (see spmm.cu)
  void* stenJ[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
  // float64 stencil copy of K for the coupled residual (grid operators; built
  // on first use after K's values change)
  double* stenK = nullptr;
  bool stenK_valid = false;
  pint::IluState* ilu = nullptr;
  pint::KrylovWork* work = nullptr;
  // nonlinear problem that owns this operator (or nullptr)
  pint_problem owner = nullptr;
};

namespace pint {

// Records (when the context's profiler is on) a CUDA event pair around the
// launches made in its scope and books algorithmic bytes / flops to `fam`.
// Raise a kernel's dynamic shared-memory limit only when a launch needs more
// than was set before (per kernel and device): the attribute call is a host
// round trip on every launch otherwise.
inline void smem_attr_raw(const void* kern, size_t bytes) {
  // the default limit (48 KB) covers static plus dynamic shared memory; the
  // library's kernels declare at most 2 KB statically
  if (bytes + 2048 <= 48 * 1024) return;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> set;
  int dev = 0;
  PINT_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = set[{kern, dev}];
  if (bytes <= cur) return;
  PINT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = bytes;
}
template <typename K>
inline void smem_attr(K* kern, size_t bytes) {
  smem_attr_raw(reinterpret_cast<const void*>(kern), bytes);
}

struct ProfScope {
  pint_ctx c;
  int fam;
  double bytes, flops;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  ProfScope(pint_ctx c_, int fam_, double bytes_, double flops_, cudaStream_t st_)
      : c(c_), fam(fam_), bytes(bytes_), flops(flops_), st(st_) {
    if (c) {
      c->prof_launches[fam] += 1;
      c->prof_bytes[fam] += bytes;
      c->prof_flops[fam] += flops;
      if (c->nvtx_on) nvtxRangePushA(family_name(fam));
    }
    if (c && c->prof_on) {
      a = take_event();
      cudaEventRecord(a, st);
    }
  }
  static const char* family_name(int f) {
    static const char* names[PF_COUNT] = {"coupled", "spmm", "gram",  "update", "cholqr",
                                          "hess",    "ilu",  "norm",  "vec",    "nl"};
    return (f >= 0 && f < PF_COUNT) ? names[f] : "other";
  }
  // nothing was launched in this scope after all: undo the counts
  void cancel() {
    if (!c) return;
    c->prof_launches[fam] -= 1;
    c->prof_bytes[fam] -= bytes;
    c->prof_flops[fam] -= flops;
    if (a) {
      c->ev_pool.push_back(a);
      a = nullptr;
    }
  }
  ~ProfScope() {
    if (c && c->nvtx_on) nvtxRangePop();
    if (c && c->prof_on && a) {
      cudaEvent_t b = take_event();
      cudaEventRecord(b, st);
      c->prof_pending.push_back({fam, a, b, bytes, flops});
    }
  }
  cudaEvent_t take_event() {
    if (!c->ev_pool.empty()) {
      cudaEvent_t e = c->ev_pool.back();
      c->ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};

// ----------------------------------------------------------- allocation
// Residual history: a solve starts a new one; each outer (or Newton)
// iteration appends its per-column relative residuals.
inline void hist_reset(pint_ctx ctx, int s) {
  ctx->hist.clear();
  ctx->hist_s = s;
}
inline void hist_push(pint_ctx ctx, const double* rel, int s) {
  if (ctx->hist_s != s) hist_reset(ctx, s);
  if (ctx->hist.size() < (size_t)1 << 22) ctx->hist.insert(ctx->hist.end(), rel, rel + s);
}

void* dalloc(pint_ctx ctx, size_t bytes);
void dfree(pint_ctx ctx, void* p, size_t bytes);
template <typename T>
T* dalloc_n(pint_ctx ctx, size_t n) { return static_cast<T*>(dalloc(ctx, n * sizeof(T))); }

// ------------------------------------------------------------ spmm.cu
void sell_build(pint_op op);                 // pattern -> SELL (device)
void sell_scatter(pint_op op, const double* csr_vals, double* sell_vals, cudaStream_t st);
void build_inner(pint_op op, cudaStream_t st);  // Jval, Jdiag, Jinvdiag
void* inner_sell(pint_op op, int precision, bool jacobi, cudaStream_t st);
int coupling_band(const double* A1, const double* A2, int s);   // 16-pitch matrices
void launch_coupled(pint_op op, const double* Y, const double* B, const double* B0,
                    double* R, cudaStream_t st);
// Z = Jsell X   (mode 0)  or  Z = Rin - Jsell X  (mode 1)
void launch_inner_spmm(pint_op op, int precision, bool jacobi, const void* X, void* Z,
                       const void* Rin, cudaStream_t st);
void launch_colnorm(pint_ctx ctx, int precision, int64_t n, int s, const void* X,
                    double* out_dev, cudaStream_t st);   // out_dev[k] = ||X_k||_2
// Y -= diag(scale) * Dinv? * V  (float64 Y; V float64 or float32)
void launch_outer_update(int precision, int64_t n, int s, double* Y, const void* V,
                         const double* colscale, const double* rowscale, cudaStream_t st,
                         pint_ctx ctx, int ys = 0, int yoff = 0);
void launch_gather_cols(int64_t n, int s, int c0, int w, const double* src, double* dst,
                        cudaStream_t st, pint_ctx ctx);
// dst(float32) = src(float64) * 1/colscale[k]
void launch_scale_cast(int64_t n, int s, const double* src, float* dst,
                       const double* inv_colscale, cudaStream_t st, pint_ctx ctx);
void launch_scale_copy64(int64_t n, int s, const double* src, double* dst,
                         const double* inv_colscale, cudaStream_t st, pint_ctx ctx);
void launch_copy_cast(int precision, int64_t n, int s, const double* src, void* dst,
                      cudaStream_t st, pint_ctx ctx);
void launch_shift(double* Y, int64_t n, int s, cudaStream_t st, pint_ctx ctx);
// out[k] = rnorm[k] * min(1, delta / max_r |rnorm[k] rowscale[r] X[r][k]|)
void launch_step_bound(int precision, int64_t n, int s, const void* X, const double* rowscale,
                       const double* rnorm, double delta, double* out, cudaStream_t st,
                       pint_ctx ctx);

// ----------------------------------------------------------- krylov.cu
// n_pad > 0: rows [n, n_pad) of V and W are zero and n_pad % 64 == 0, which
// enables the bulk-copy (TMA) pipeline; 0: plain loads.
void launch_gram(pint_ctx ctx, int precision, int64_t n, int s, int nb, const void* V,
                 int64_t bstride, const void* W, double* H, cudaStream_t st, int64_t n_pad = 0);
// mode 0: W -= V H ; 1: W = V H ; 2: W += V H
void launch_update(pint_ctx ctx, int precision, int64_t n, int s, int nb, const void* V,
                   int64_t bstride, const double* H, void* W, int mode, cudaStream_t st);
void cholqr2(pint_ctx ctx, int precision, int64_t n, int s, void* W, double* R,
             int* defl_count_dev, cudaStream_t st, int64_t n_pad = 0);
int solve_block_impl(pint_op op, const double* B, const double* B0, double* Y,
                     const pint_opts* o, pint_stats* stats, cudaStream_t st);
// Inner solve J V = R (R float64, scaled per column inside), result V float64.
// Returns number of Arnoldi steps; throws on failure.
struct InnerResult { int its; int cycles; bool converged; int deflations; };
InnerResult inner_solve(pint_op op, const pint_opts* o, const double* R, const double* rnorm_host,
                        double* V, cudaStream_t st);

void work_views(pint_op op, int prec, int m, double** R64, double** rnorm, void** Xk,
                int* wprec);
// api.cu: operator with a host CSR pattern and zero values
pint_op op_create(pint_ctx ctx, int64_t n, const int* rowptr, const int* colind,
                  cudaStream_t st);
void op_free_all(pint_op op);
void op_clear_inner_cache(pint_op op);

// -------------------------------------------------------------- ilu.cu
void ilu_setup(pint_op op, cudaStream_t st);          // factor J (float64 + float32 copy)
void ilu_apply(pint_op op, int precision, const void* X, void* Z, cudaStream_t st);
void ilu_destroy(pint_op op);
void ilu_check(pint_op op);                            // throws PINT_ERR_TIMEOUT
// Bounded waits made to run out (test access): the ILU(0) dependency wait on
// a flag nothing sets, and the Gram ring's mbarrier wait on a transaction
// count no copy delivers. Each raises its error word and returns.
void test_wait_timeout(double limit_ms, unsigned* flag, int* err, cudaStream_t st);
void test_mbar_timeout(double limit_ms, int* err, cudaStream_t st);

}  // namespace pint

#include <type_traits>
namespace pint {
// Dispatch a runtime block width s (1..16) to a compile-time (S, EXACT) pair:
// s in {1,2,4,8,16} runs the exact, vectorised instantiation; other widths run
// the next power of two with guarded loads.
template <typename Fn>
void with_s(int s, Fn&& fn) {
  using T = std::true_type;
  using F = std::false_type;
  switch (s) {
    case 1: fn(std::integral_constant<int, 1>{}, T{}); break;
    case 2: fn(std::integral_constant<int, 2>{}, T{}); break;
    case 3: fn(std::integral_constant<int, 4>{}, F{}); break;
    case 4: fn(std::integral_constant<int, 4>{}, T{}); break;
    case 5: case 6: case 7: fn(std::integral_constant<int, 8>{}, F{}); break;
    case 8: fn(std::integral_constant<int, 8>{}, T{}); break;
    case 16: fn(std::integral_constant<int, 16>{}, T{}); break;
    default:
      if (s >= 9 && s <= 15) fn(std::integral_constant<int, 16>{}, F{});
      else throw Error{PINT_ERR_INVALID, "block width s must be in 1..16"};
  }
}
inline unsigned grid_for(int64_t n, int threads) {
  return static_cast<unsigned>((n + threads - 1) / threads);
}
}  // namespace pint
