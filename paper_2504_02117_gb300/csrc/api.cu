// C ABI of libpint: contexts, device-memory accounting, operators, coupling,
// and the exposed building blocks. Every entry point converts exceptions into
// a status code and records the message in the context.
#include "internal.h"

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <mutex>

namespace pint {

void free_work(pint_op op);   // krylov.cu

void* dalloc(pint_ctx ctx, size_t bytes) {
  if (bytes == 0) bytes = 16;
  PINT_REQUIRE(ctx->used + bytes <= ctx->budget, PINT_ERR_NOMEM,
               "device memory budget exceeded (" + std::to_string(ctx->used + bytes) + " > " +
                   std::to_string(ctx->budget) + " bytes)");
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error{PINT_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
  }
  ctx->used += bytes;
  return p;
}

void dfree(pint_ctx ctx, void* p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  cudaFree(p);
  ctx->used -= std::min(ctx->used, bytes);
}

static thread_local std::string g_noctx_err;
void set_noctx_error(const std::string& msg) { g_noctx_err = msg; }

template <typename Fn>
static int guard(pint_ctx ctx, Fn&& fn) {
  try {
    if (ctx) PINT_CUDA(cudaSetDevice(ctx->device));
    return fn();
  } catch (const Error& e) {
    if (ctx) ctx->err = e.msg; else g_noctx_err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->err = "host allocation failed"; else g_noctx_err = "host allocation failed";
    return PINT_ERR_NOMEM;
  } catch (...) {
    if (ctx) ctx->err = "unknown error"; else g_noctx_err = "unknown error";
    return PINT_ERR_INVALID;
  }
}

static inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

static void require_aligned(const void* p, const char* name) {
  PINT_REQUIRE(reinterpret_cast<uintptr_t>(p) % 16 == 0, PINT_ERR_INVALID,
               std::string(name) + " must be 16-byte aligned");
}

void op_clear_inner_cache(pint_op op);

// Copy the CSR pattern to host (validating it) and build device structures.
static void op_build_pattern(pint_op op, const int32_t* rowptr, const int32_t* colind,
                             int mem_space) {
  const int64_t n = op->n;
  op->h_rowptr.resize(n + 1);
  if (mem_space == PINT_MEM_DEVICE)
    PINT_CUDA(cudaMemcpy(op->h_rowptr.data(), rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost));
  else
    std::memcpy(op->h_rowptr.data(), rowptr, sizeof(int) * (n + 1));
  PINT_REQUIRE(op->h_rowptr[0] == 0, PINT_ERR_INVALID, "rowptr[0] must be 0");
  for (int64_t r = 0; r < n; ++r)
    PINT_REQUIRE(op->h_rowptr[r + 1] >= op->h_rowptr[r], PINT_ERR_INVALID, "rowptr not monotone");
  op->nnz = op->h_rowptr[n];
  op->h_colind.resize(std::max<int64_t>(op->nnz, 1));
  if (mem_space == PINT_MEM_DEVICE)
    PINT_CUDA(cudaMemcpy(op->h_colind.data(), colind, sizeof(int) * op->nnz, cudaMemcpyDeviceToHost));
  else
    std::memcpy(op->h_colind.data(), colind, sizeof(int) * op->nnz);
  std::vector<int> dpos(n);
  for (int64_t r = 0; r < n; ++r) {
    int d = -1;
    for (int p = op->h_rowptr[r]; p < op->h_rowptr[r + 1]; ++p) {
      const int c = op->h_colind[p];
      PINT_REQUIRE(c >= 0 && c < n, PINT_ERR_INVALID, "column index out of range");
      if (p > op->h_rowptr[r])
        PINT_REQUIRE(c > op->h_colind[p - 1], PINT_ERR_INVALID,
                     "column indices must be strictly increasing in each row");
      if (c == r) d = p;
    }
    PINT_REQUIRE(d >= 0, PINT_ERR_INVALID, "every row needs a diagonal entry");
    dpos[r] = d;
  }
  op->rowptr = dalloc_n<int>(op->ctx, n + 1);
  op->colind = dalloc_n<int>(op->ctx, std::max<int64_t>(op->nnz, 1));
  op->diagpos = dalloc_n<int>(op->ctx, n);
  PINT_CUDA(cudaMemcpy(op->rowptr, op->h_rowptr.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
  PINT_CUDA(cudaMemcpy(op->colind, op->h_colind.data(), sizeof(int) * op->nnz, cudaMemcpyHostToDevice));
  PINT_CUDA(cudaMemcpy(op->diagpos, dpos.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  sell_build(op);
  op->Kval = dalloc_n<double>(op->ctx, std::max<int64_t>(op->nnz, 1));
  op->sellK = dalloc_n<double>(op->ctx, std::max<int64_t>(op->sell.nelem, 1));
}

static void op_set_values(pint_op op, const double* K, const double* M, int mem_space,
                          cudaStream_t st) {
  const cudaMemcpyKind kind =
      mem_space == PINT_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (K) {
    PINT_CUDA(cudaMemcpyAsync(op->Kval, K, sizeof(double) * op->nnz, kind, st));
    sell_scatter(op, op->Kval, op->sellK, st);
  }
  if (M) {
    if (!op->Mdiag) op->Mdiag = dalloc_n<double>(op->ctx, op->n);
    PINT_CUDA(cudaMemcpyAsync(op->Mdiag, M, sizeof(double) * op->n, kind, st));
  }
  op_clear_inner_cache(op);
  op->j_valid = false;
}

pint_op op_create(pint_ctx ctx, int64_t n, const int* rowptr, const int* colind,
                  cudaStream_t st) {
  pint_op op = new pint_op_s();
  op->ctx = ctx;
  op->n = n;
  try {
    op_build_pattern(op, rowptr, colind, PINT_MEM_HOST);
    PINT_CUDA(cudaMemsetAsync(op->Kval, 0, sizeof(double) * std::max<int64_t>(op->nnz, 1), st));
    PINT_CUDA(cudaMemsetAsync(op->sellK, 0, sizeof(double) * std::max<int64_t>(op->sell.nelem, 1), st));
  } catch (...) {
    op_free_all(op);
    delete op;
    throw;
  }
  return op;
}

void op_free_all(pint_op op) {
  pint_ctx c = op->ctx;
  free_work(op);
  if (op->ilu) ilu_destroy(op);
  const int64_t n = op->n, nnz = std::max<int64_t>(op->nnz, 1);
  const int64_t ne = std::max<int64_t>(op->sell.nelem, 1);
  const size_t esz[3] = {8, 4, 2};
  for (int p = 0; p < 3; ++p)
    for (int j = 0; j < 2; ++j) {
      if (op->sellJ[p][j]) dfree(c, op->sellJ[p][j], esz[p] * op->sell.nelem);
      if (op->stenJ[p][j]) dfree(c, op->stenJ[p][j], esz[p] * 8 * op->n);
    }
  dfree(c, op->rowptr, sizeof(int) * (n + 1));
  dfree(c, op->colind, sizeof(int) * nnz);
  dfree(c, op->diagpos, sizeof(int) * n);
  dfree(c, op->Kval, sizeof(double) * nnz);
  dfree(c, op->sellK, sizeof(double) * ne);
  dfree(c, op->stenK, sizeof(double) * 8 * n);
  dfree(c, op->Mdiag, sizeof(double) * n);
  dfree(c, op->Jval, sizeof(double) * nnz);
  dfree(c, op->Jdiag, sizeof(double) * n);
  dfree(c, op->Jinvdiag, sizeof(double) * n);
  dfree(c, op->sell.slice_ptr, sizeof(int64_t) * (op->sell.nslices + 1));
  dfree(c, op->sell.col, sizeof(int) * ne);
  dfree(c, op->sell.csr_to_sell, sizeof(int64_t) * nnz);
}

void op_clear_inner_cache(pint_op op) {
  const size_t esz[3] = {8, 4, 2};
  for (int p = 0; p < 3; ++p)
    for (int j = 0; j < 2; ++j) {
      if (op->sellJ[p][j]) {
        dfree(op->ctx, op->sellJ[p][j], esz[p] * op->sell.nelem);
        op->sellJ[p][j] = nullptr;
      }
      if (op->stenJ[p][j]) {
        dfree(op->ctx, op->stenJ[p][j], esz[p] * 8 * op->n);
        op->stenJ[p][j] = nullptr;
      }
    }
  if (op->ilu) ilu_destroy(op);
}

__global__ void k_rowscale(int64_t n, int s, const double* __restrict__ X,
                           const double* __restrict__ d, double* __restrict__ Z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * s) Z[i] = X[i] * d[i / s];
}

}  // namespace pint

using namespace pint;

// ================================================================= C ABI
extern "C" {

void pint_opts_default(pint_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-10;
  o->inner_tol = 1e-2;
  o->restart = 30;
  o->max_outer = 200;
  o->max_inner = 3000;
  o->precond = PINT_PC_JACOBI;
  o->precision = PINT_FP64;
}

int pint_create(pint_ctx* out, int device, size_t budget) {
  if (!out) return PINT_ERR_INVALID;
  *out = nullptr;
  pint_ctx ctx = new pint_ctx_s();
  ctx->device = device;
  int rc = guard(ctx, [&] {
    cudaDeviceProp prop;
    PINT_CUDA(cudaGetDeviceProperties(&prop, device));
    ctx->num_sms = prop.multiProcessorCount;
    size_t fr = 0, tot = 0;
    PINT_CUDA(cudaMemGetInfo(&fr, &tot));
    ctx->budget = budget ? budget : (size_t)(0.9 * (double)fr);
    const char* fz = std::getenv("PINT_GRAM_FUSE");
    ctx->gram_fuse = !(fz && fz[0] == '0');
    PINT_CUDA(cudaMallocHost(&ctx->h_flag, 64 * sizeof(int)));
    PINT_CUDA(cudaMallocHost(&ctx->h_small, 4096 * sizeof(double)));
    ctx->d_small = dalloc_n<double>(ctx, kSmallDoubles);
    ctx->d_flag = dalloc_n<int>(ctx, 64);
    PINT_CUDA(cudaMemset(ctx->d_small, 0, sizeof(double) * kSmallDoubles));
    PINT_CUDA(cudaMemset(ctx->d_flag, 0, 64 * sizeof(int)));    // device error words
    return PINT_OK;
  });
  if (rc != PINT_OK) {
    g_noctx_err = ctx->err;
    if (ctx->h_flag) cudaFreeHost(ctx->h_flag);
    if (ctx->h_small) cudaFreeHost(ctx->h_small);
    delete ctx;
    return rc;
  }
  *out = ctx;
  return PINT_OK;
}

int pint_destroy(pint_ctx ctx) {
  if (!ctx) return PINT_ERR_INVALID;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& r : ctx->prof_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  dfree(ctx, ctx->d_small, sizeof(double) * kSmallDoubles);
  dfree(ctx, ctx->d_flag, 64 * sizeof(int));
  dfree(ctx, ctx->d_partial, ctx->partial_bytes);
  if (ctx->h_flag) cudaFreeHost(ctx->h_flag);
  if (ctx->h_small) cudaFreeHost(ctx->h_small);
  delete ctx;
  return PINT_OK;
}

const char* pint_last_error(pint_ctx ctx) {
  return ctx ? ctx->err.c_str() : g_noctx_err.c_str();
}

size_t pint_bytes_in_use(pint_ctx ctx) { return ctx ? ctx->used : 0; }

int pint_operator_assemble(pint_ctx ctx, pint_op* out, int64_t n, const int32_t* rowptr,
                           const int32_t* colind, const double* K_vals, const double* M_diag,
                           int mem_space, void* stream) {
  if (!ctx || !out) return PINT_ERR_INVALID;
  *out = nullptr;
  pint_op op = new pint_op_s();
  op->ctx = ctx;
  op->n = n;
  int rc = guard(ctx, [&] {
    PINT_REQUIRE(n >= 1 && n < (int64_t)1 << 31, PINT_ERR_INVALID, "n out of range");
    PINT_REQUIRE(rowptr && colind && K_vals, PINT_ERR_INVALID, "NULL CSR array");
    PINT_REQUIRE(mem_space == PINT_MEM_HOST || mem_space == PINT_MEM_DEVICE, PINT_ERR_INVALID,
                 "mem_space");
    op_build_pattern(op, rowptr, colind, mem_space);
    op_set_values(op, K_vals, M_diag, mem_space, as_stream(stream));
    PINT_CUDA(cudaStreamSynchronize(as_stream(stream)));
    return PINT_OK;
  });
  if (rc != PINT_OK) {
    op_free_all(op);
    delete op;
    return rc;
  }
  *out = op;
  return PINT_OK;
}

int pint_operator_update_values(pint_op op, const double* K_vals, const double* M_diag,
                                int mem_space, void* stream) {
  if (!op) return PINT_ERR_INVALID;
  return guard(op->ctx, [&] {
    op_clear_inner_cache(op);
    op_set_values(op, K_vals, M_diag, mem_space, as_stream(stream));
    PINT_CUDA(cudaStreamSynchronize(as_stream(stream)));
    return PINT_OK;
  });
}

int pint_operator_destroy(pint_op op) {
  if (!op) return PINT_ERR_INVALID;
  cudaSetDevice(op->ctx->device);
  op_free_all(op);
  delete op;
  return PINT_OK;
}

int64_t pint_operator_nnz(pint_op op) { return op ? op->nnz : -1; }

int pint_set_coupling(pint_op op, int s, const double* A1, const double* A2) {
  if (!op) return PINT_ERR_INVALID;
  return guard(op->ctx, [&] {
    PINT_REQUIRE(s >= 1 && s <= PINT_MAX_S, PINT_ERR_INVALID, "s must be in 1..16");
    PINT_REQUIRE(A1 && A2, PINT_ERR_INVALID, "NULL coupling matrix");
    for (int i = 0; i < s * s; ++i)
      PINT_REQUIRE(std::isfinite(A1[i]) && std::isfinite(A2[i]), PINT_ERR_INVALID,
                   "non-finite coupling entry");
    PINT_REQUIRE(A1[0] != 0.0 || A2[0] != 0.0, PINT_ERR_INVALID,
                 "alpha = A1[0][0] and beta = A2[0][0] are both zero");
    std::fill(op->A1, op->A1 + kMaxS * kMaxS, 0.0);
    std::fill(op->A2, op->A2 + kMaxS * kMaxS, 0.0);
    for (int i = 0; i < s; ++i)
      for (int k = 0; k < s; ++k) {
        op->A1[i * kMaxS + k] = A1[i * s + k];
        op->A2[i * kMaxS + k] = A2[i * s + k];
      }
    const double a = A1[0], b = A2[0];
    if (a != op->alpha || b != op->beta) {
      op_clear_inner_cache(op);
      op->j_valid = false;
    }
    if (s != op->s) free_work(op);
    op->alpha = a;
    op->beta = b;
    op->s = s;
    return PINT_OK;
  });
}

int pint_coupling_from_dirk(const double* A, int m, int steps, double tau, int eliminate_first,
                            double* A1, double* A2, double* e, int* s_out) {
  return guard(nullptr, [&] {
    PINT_REQUIRE(A && A1 && A2 && s_out && m >= 1 && steps >= 1 && tau > 0.0, PINT_ERR_INVALID,
                 "bad arguments");
    const int mp = eliminate_first ? m - 1 : m;
    PINT_REQUIRE(mp >= 1, PINT_ERR_INVALID, "nothing left after elimination");
    if (eliminate_first)
      for (int j = 0; j < m; ++j)
        PINT_REQUIRE(A[j] == 0.0, PINT_ERR_INVALID, "first stage is not explicit");
    const int S = steps * mp;
    PINT_REQUIRE(S <= PINT_MAX_S, PINT_ERR_INVALID, "steps * stages exceeds 16");
    const int off = eliminate_first ? 1 : 0;
    std::fill(A1, A1 + S * S, 0.0);
    std::fill(A2, A2 + S * S, 0.0);
    for (int nblk = 0; nblk < steps; ++nblk)
      for (int i = 0; i < mp; ++i) {
        const int r = nblk * mp + i;
        A1[r * S + r] = 1.0 / tau;
        for (int j = 0; j < mp; ++j) A2[r * S + nblk * mp + j] = A[(i + off) * m + (j + off)];
        if (nblk > 0) {
          const int last = nblk * mp - 1;
          A1[r * S + last] = -1.0 / tau;
          if (eliminate_first) A2[r * S + last] = A[(i + off) * m + 0];
        }
      }
    if (e && eliminate_first)
      for (int i = 0; i < mp; ++i) e[i] = A[(i + 1) * m];
    *s_out = S;
    return PINT_OK;
  });
}

int pint_apply_coupled(pint_op op, const double* Y, const double* B, const double* B0, double* R,
                       void* stream) {
  if (!op) return PINT_ERR_INVALID;
  return guard(op->ctx, [&] {
    PINT_REQUIRE(op->s >= 1, PINT_ERR_INVALID, "coupling not set");
    PINT_REQUIRE(Y && R, PINT_ERR_INVALID, "NULL Y or R");
    require_aligned(Y, "Y");
    require_aligned(R, "R");
    if (B) require_aligned(B, "B");
    if (B0) require_aligned(B0, "B0");
    launch_coupled(op, Y, B, B0, R, as_stream(stream));
    return PINT_OK;
  });
}

int pint_solve_block(pint_op op, const double* B, const double* B0, double* Y,
                     const pint_opts* opts, pint_stats* stats, void* stream) {
  if (!op) return PINT_ERR_INVALID;
  pint_opts o;
  if (opts) o = *opts; else pint_opts_default(&o);
  if (stats) std::memset(stats, 0, sizeof(*stats));
  int rc = guard(op->ctx, [&] {
    PINT_REQUIRE(Y, PINT_ERR_INVALID, "NULL Y");
    require_aligned(Y, "Y");
    if (B) require_aligned(B, "B");
    if (B0) require_aligned(B0, "B0");
    return solve_block_impl(op, B, B0, Y, &o, stats, as_stream(stream));
  });
  if (stats) stats->status = rc;
  return rc;
}

int pint_shift(double* Y, int64_t n, int s, void* stream) {
  return guard(nullptr, [&] {
    PINT_REQUIRE(Y && n >= 0 && s >= 1 && s <= PINT_MAX_S, PINT_ERR_INVALID, "bad arguments");
    if (n > 0 && s > 1) launch_shift(Y, n, s, as_stream(stream), nullptr);
    return PINT_OK;
  });
}

int pint_inner_apply(pint_op op, const double* X, double* Z, void* stream) {
  if (!op) return PINT_ERR_INVALID;
  return guard(op->ctx, [&] {
    PINT_REQUIRE(op->s >= 1, PINT_ERR_INVALID, "coupling not set");
    require_aligned(X, "X");
    require_aligned(Z, "Z");
    cudaStream_t st = as_stream(stream);
    if (!op->j_valid) build_inner(op, st);
    launch_inner_spmm(op, PINT_FP64, false, X, Z, nullptr, st);
    return PINT_OK;
  });
}

int pint_inner_apply_lowp(pint_op op, int precision, const float* X, float* Z, void* stream) {
  if (!op) return PINT_ERR_INVALID;
  return guard(op->ctx, [&] {
    PINT_REQUIRE(op->s >= 1, PINT_ERR_INVALID, "coupling not set");
    PINT_REQUIRE(precision == PINT_FP32 || precision == PINT_BF16, PINT_ERR_INVALID,
                 "precision must be PINT_FP32 or PINT_BF16");
    require_aligned(X, "X");
    require_aligned(Z, "Z");
    PINT_REQUIRE(X != Z, PINT_ERR_INVALID, "X and Z must not alias");
    cudaStream_t st = as_stream(stream);
    if (!op->j_valid) build_inner(op, st);
    launch_inner_spmm(op, precision, false, X, Z, nullptr, st);
    return PINT_OK;
  });
}

int pint_ilu0_apply_f32(pint_op op, const float* X, float* Z, void* stream) {
  if (!op) return PINT_ERR_INVALID;
  return guard(op->ctx, [&] {
    PINT_REQUIRE(op->s >= 1, PINT_ERR_INVALID, "coupling not set");
    require_aligned(X, "X");
    require_aligned(Z, "Z");
    PINT_REQUIRE(X != Z, PINT_ERR_INVALID, "X and Z must not alias");
    cudaStream_t st = as_stream(stream);
    if (!op->j_valid) build_inner(op, st);
    ilu_setup(op, st);
    ilu_apply(op, PINT_FP32, X, Z, st);
    PINT_CUDA(cudaStreamSynchronize(st));
    ilu_check(op);
    return PINT_OK;
  });
}

int pint_precond_apply(pint_op op, int precond, const double* X, double* Z, void* stream) {
  if (!op) return PINT_ERR_INVALID;
  return guard(op->ctx, [&] {
    PINT_REQUIRE(op->s >= 1, PINT_ERR_INVALID, "coupling not set");
    require_aligned(X, "X");
    require_aligned(Z, "Z");
    PINT_REQUIRE(X != Z, PINT_ERR_INVALID, "X and Z must not alias");
    cudaStream_t st = as_stream(stream);
    if (!op->j_valid) build_inner(op, st);
    const int64_t ne = op->n * op->s;
    if (precond == PINT_PC_NONE) {
      PINT_CUDA(cudaMemcpyAsync(Z, X, sizeof(double) * ne, cudaMemcpyDeviceToDevice, st));
    } else if (precond == PINT_PC_JACOBI) {
      k_rowscale<<<grid_for(ne, 256), 256, 0, st>>>(op->n, op->s, X, op->Jinvdiag, Z);
      check_launch("k_rowscale");
    } else if (precond == PINT_PC_ILU0) {
      ilu_setup(op, st);
      ilu_apply(op, PINT_FP64, X, Z, st);
      PINT_CUDA(cudaStreamSynchronize(st));
      ilu_check(op);
    } else {
      throw Error{PINT_ERR_INVALID, "precond"};
    }
    return PINT_OK;
  });
}

int pint_block_gram(pint_ctx ctx, int precision, int64_t n, int s, int nb, const void* V,
                    const void* W, double* H, void* stream) {
  if (!ctx) return PINT_ERR_INVALID;
  return guard(ctx, [&] {
    PINT_REQUIRE(n >= 1 && s >= 1 && s <= PINT_MAX_S && nb >= 1, PINT_ERR_INVALID, "sizes");
    PINT_REQUIRE(precision == PINT_FP64 || precision == PINT_FP32, PINT_ERR_INVALID, "precision");
    require_aligned(V, "V");
    require_aligned(W, "W");
    cudaStream_t st = as_stream(stream);
    // the bulk-copy pipeline raises the context's error word when a wait runs
    // out: clear it first, read it after the product
    PINT_CUDA(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), st));
    // n a multiple of 64 needs no padding rows: use the bulk-copy pipeline
    launch_gram(ctx, precision, n, s, nb, V, n * s, W, H, st, n % 64 == 0 ? n : 0);
    PINT_CUDA(cudaMemcpyAsync(ctx->h_flag + 2, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    PINT_CUDA(cudaStreamSynchronize(st));
    PINT_REQUIRE(ctx->h_flag[2] == 0, PINT_ERR_TIMEOUT,
                 "bulk-copy wait in the Gram kernel exceeded its time budget");
    return PINT_OK;
  });
}

int pint_block_update(pint_ctx ctx, int precision, int64_t n, int s, int nb, const void* V,
                      const double* H, void* W, void* stream) {
  if (!ctx) return PINT_ERR_INVALID;
  return guard(ctx, [&] {
    PINT_REQUIRE(n >= 1 && s >= 1 && s <= PINT_MAX_S && nb >= 1 && nb * s <= 1024,
                 PINT_ERR_INVALID, "sizes");
    PINT_REQUIRE(precision == PINT_FP64 || precision == PINT_FP32, PINT_ERR_INVALID, "precision");
    require_aligned(V, "V");
    require_aligned(W, "W");
    launch_update(ctx, precision, n, s, nb, V, n * s, H, W, 0, as_stream(stream));
    return PINT_OK;
  });
}

int pint_cholqr2(pint_ctx ctx, int precision, int64_t n, int s, void* W, double* R,
                 void* stream) {
  if (!ctx) return PINT_ERR_INVALID;
  return guard(ctx, [&] {
    PINT_REQUIRE(n >= 1 && s >= 1 && s <= PINT_MAX_S, PINT_ERR_INVALID, "sizes");
    PINT_REQUIRE(precision == PINT_FP64 || precision == PINT_FP32, PINT_ERR_INVALID, "precision");
    require_aligned(W, "W");
    cholqr2(ctx, precision, n, s, W, R, nullptr, as_stream(stream));
    return PINT_OK;
  });
}

// Eight independent float64 FMA chains per thread (latency hidden), one
// result per thread so nothing is optimised away.
__global__ void __launch_bounds__(256) k_fp64_fma_peak(int iters, double* out) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1e-3 * (threadIdx.x + k);
  const double b = 0.9999999, c = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  double v = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) v += a[k];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = v;
}

int pint_fp64_fma_peak(pint_ctx ctx, double* tflops) {
  if (!ctx || !tflops) return PINT_ERR_INVALID;
  return guard(ctx, [&] {
    const int blocks = ctx->num_sms * 8, threads = 256, iters = 4096;
    double* out = dalloc_n<double>(ctx, (size_t)blocks * threads);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = 0.0;
    try {
      PINT_CUDA(cudaEventCreate(&e0));
      PINT_CUDA(cudaEventCreate(&e1));
      for (int rep = 0; rep < 4; ++rep) {            // the first is a warm-up
        PINT_CUDA(cudaEventRecord(e0, nullptr));
        k_fp64_fma_peak<<<blocks, threads>>>(iters, out);
        check_launch("k_fp64_fma_peak");
        PINT_CUDA(cudaEventRecord(e1, nullptr));
        PINT_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        PINT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        const double fl = 2.0 * 8.0 * iters * (double)blocks * threads;
        if (rep > 0 && ms > 0.f) best = std::max(best, fl / (ms * 1e-3) / 1e12);
      }
      ctx->launches += 4;
    } catch (...) {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      dfree(ctx, out, sizeof(double) * blocks * threads);
      throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(ctx, out, sizeof(double) * blocks * threads);
    *tflops = best;
    return PINT_OK;
  });
}

int pint_test_wait_timeout(pint_ctx ctx, int which, double limit_ms, void* stream) {
  if (!ctx) return PINT_ERR_INVALID;
  return guard(ctx, [&] {
    PINT_REQUIRE(which == 0 || which == 1, PINT_ERR_INVALID, "which must be 0 or 1");
    PINT_REQUIRE(limit_ms > 0.0 && limit_ms <= 1000.0, PINT_ERR_INVALID,
                 "limit_ms must be in (0, 1000]");
    cudaStream_t st = as_stream(stream);
    // words 8 (a flag nothing sets) and 9 (the error word) of the context's
    // flag array, which no solve uses
    unsigned* flag = reinterpret_cast<unsigned*>(ctx->d_flag + 8);
    int* err = ctx->d_flag + 9;
    PINT_CUDA(cudaMemsetAsync(ctx->d_flag + 8, 0, 2 * sizeof(int), st));
    if (which == 0) test_wait_timeout(limit_ms, flag, err, st);
    else test_mbar_timeout(limit_ms, err, st);
    ctx->launches += 1;
    PINT_CUDA(cudaMemcpyAsync(ctx->h_flag + 3, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    PINT_CUDA(cudaStreamSynchronize(st));
    const int e = ctx->h_flag[3];
    PINT_REQUIRE(e == 0, PINT_ERR_TIMEOUT,
                 which == 0 ? "ILU(0) dependency wait exceeded its time budget"
                            : "bulk-copy (mbarrier) wait exceeded its time budget");
    return PINT_OK;
  });
}

int pint_colnorms(pint_ctx ctx, int precision, int64_t n, int s, const void* X, double* norms,
                  void* stream) {
  if (!ctx) return PINT_ERR_INVALID;
  return guard(ctx, [&] {
    PINT_REQUIRE(n >= 1 && s >= 1 && s <= PINT_MAX_S && norms, PINT_ERR_INVALID, "sizes");
    PINT_REQUIRE(precision == PINT_FP64 || precision == PINT_FP32, PINT_ERR_INVALID, "precision");
    require_aligned(X, "X");
    cudaStream_t st = as_stream(stream);
    double* d = ctx->d_small + kSmallScratch;
    launch_colnorm(ctx, precision, n, s, X, d, st);
    PINT_CUDA(cudaMemcpyAsync(ctx->h_small, d, 8 * s, cudaMemcpyDeviceToHost, st));
    PINT_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < s; ++k) norms[k] = ctx->h_small[k];
    return PINT_OK;
  });
}

}  // extern "C"

// ------------------------------------------------------------- profiler
namespace pint {
static void prof_collect(pint_ctx ctx) {
  if (ctx->prof_pending.empty()) return;
  PINT_CUDA(cudaDeviceSynchronize());
  for (auto& r : ctx->prof_pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) ctx->prof_ms[r.fam] += ms;
    ctx->ev_pool.push_back(r.a);
    ctx->ev_pool.push_back(r.b);
  }
  ctx->prof_pending.clear();
}
}  // namespace pint

extern "C" {

int pint_profile_enable(pint_ctx ctx, int on) {
  if (!ctx) return PINT_ERR_INVALID;
  return guard(ctx, [&] {
    PINT_REQUIRE(on >= 0 && on <= 3, PINT_ERR_INVALID, "profile flags: 0..3");
    ctx->prof_on = (on & 1) != 0;
    ctx->nvtx_on = (on & 2) != 0;
    return PINT_OK;
  });
}

int pint_residual_history(pint_ctx ctx, double* out, int max_rows, int* rows, int* s) {
  if (!ctx) return PINT_ERR_INVALID;
  return guard(ctx, [&] {
    PINT_REQUIRE(max_rows >= 0, PINT_ERR_INVALID, "max_rows < 0");
    const int w = ctx->hist_s;
    const int nr = w > 0 ? (int)(ctx->hist.size() / w) : 0;
    if (rows) *rows = nr;
    if (s) *s = w;
    if (out && w > 0) {
      const int k = std::min(nr, max_rows);
      std::copy(ctx->hist.begin(), ctx->hist.begin() + (size_t)k * w, out);
    }
    return PINT_OK;
  });
}

namespace {
// Evaluates one index check of the checked build (site 99) and nothing else:
// no memory is accessed through the index, in either build.
__global__ void k_test_bounds(long long i, long long n, int* sink) {
  if (PINT_INDEX_OK(i, n, 99) && sink) *sink = 1;
}
}  // namespace

int pint_test_bounds(pint_ctx ctx, long long index, long long bound) {
  if (!ctx) return PINT_ERR_INVALID;
  return guard(ctx, [&] {
    k_test_bounds<<<1, 1>>>(index, bound, nullptr);
    check_launch("k_test_bounds");
    PINT_CUDA(cudaDeviceSynchronize());
    return PINT_OK;
  });
}

int pint_bounds_report(pint_ctx ctx, long long* count, int* site, long long* index,
                       long long* bound) {
  if (!ctx) return PINT_ERR_INVALID;
  return guard(ctx, [&] {
    PINT_CUDA(cudaDeviceSynchronize());
#ifdef PINT_BOUNDS
    unsigned long long rec[3][4];
    pint_bounds_take(rec[0]);
    bounds_take_spmm(rec[1]);
    bounds_take_batch(rec[2]);
    long long n = 0;
    int first = -1;
    for (int t = 0; t < 3; ++t) {
      n += (long long)rec[t][0];
      if (first < 0 && rec[t][0] > 0) first = t;
    }
    if (count) *count = n;
    if (site) *site = first >= 0 ? (int)rec[first][1] : 0;
    if (index) *index = first >= 0 ? (long long)rec[first][2] : 0;
    if (bound) *bound = first >= 0 ? (long long)rec[first][3] : 0;
#else
    if (count) *count = -1;
    if (site) *site = 0;
    if (index) *index = 0;
    if (bound) *bound = 0;
#endif
    return PINT_OK;
  });
}

int pint_residual_history_reset(pint_ctx ctx) {
  if (!ctx) return PINT_ERR_INVALID;
  return guard(ctx, [&] {
    hist_reset(ctx, 0);
    return PINT_OK;
  });
}

int pint_profile_read(pint_ctx ctx, int k, double* ms, double* bytes, double* flops,
                      long long* launches) {
  if (!ctx) return PINT_ERR_INVALID;
  return guard(ctx, [&] {
    PINT_REQUIRE(k >= 0 && k < PF_COUNT, PINT_ERR_INVALID, "kernel family");
    prof_collect(ctx);
    if (ms) *ms = ctx->prof_ms[k];
    if (bytes) *bytes = ctx->prof_bytes[k];
    if (flops) *flops = ctx->prof_flops[k];
    if (launches) *launches = ctx->prof_launches[k];
    return PINT_OK;
  });
}

int pint_profile_reset(pint_ctx ctx) {
  if (!ctx) return PINT_ERR_INVALID;
  return guard(ctx, [&] {
    prof_collect(ctx);
    for (int k = 0; k < PF_COUNT; ++k) {
      ctx->prof_ms[k] = ctx->prof_bytes[k] = ctx->prof_flops[k] = 0.0;
      ctx->prof_launches[k] = 0;
    }
    return PINT_OK;
  });
}

long long pint_kernel_launches(pint_ctx ctx) { return ctx ? ctx->launches : -1; }

}  // extern "C"
