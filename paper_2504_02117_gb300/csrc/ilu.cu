// ILU(0) of the inner operator J in natural row order, applied to s columns
// at once (column-batched preconditioner of the block solve).
//
// Natural-order ILU(0) (IKJ variant: for each row i and each k < i in its
// pattern, l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj for j > k in both rows'
// patterns) and its forward / backward substitutions are sequential through
// row dependencies. On the device every row waits only for the rows it reads:
//  * the host groups rows into dependency levels (level(i) = 1 + max level of
//    the rows it reads) and cuts each level into chunks of rows;
//  * warps take chunks in level order from an atomic ticket, so a chunk only
//    ever waits for chunks with lower tickets, all of which were taken by
//    running warps: the scheme cannot deadlock whatever the grid size;
//  * a finished row publishes itself by storing the launch's epoch into its
//    flag (release); readers poll with acquire loads and read finished rows
//    through L2 (ld.global.cg);
//  * every wait is bounded by a wall-clock budget (globaltimer). When it runs
//    out the kernel raises an error word; all other waits then stop at once
//    and the host reports PINT_ERR_TIMEOUT instead of a result.
#include "internal.h"

#include <algorithm>
#include <map>

namespace pint {

constexpr unsigned long long kWaitBudgetNs = 2000000000ull;   // 2 s per launch

struct Sched {
  int* order = nullptr;     // device: rows in level order
  int* chunk = nullptr;     // device: chunk start positions (nchunk + 1)
  int nchunk = 0;
  size_t bytes_chunk = 0;
};

struct IluState {
  bool factored = false;
  double* F64 = nullptr;          // factored values in the CSR pattern of J
  float* F32 = nullptr;
  unsigned* flag_f = nullptr;     // forward / factor flags
  unsigned* flag_b = nullptr;     // backward flags
  unsigned epoch_f = 0, epoch_b = 0;
  int* ticket = nullptr;          // 2 ints
  int* err = nullptr;             // device error word
  std::vector<int> order_f, lvlptr_f, order_b, lvlptr_b;
  int* d_order_f = nullptr;
  int* d_order_b = nullptr;
  std::map<int, Sched> sched_f, sched_b;   // by rows per chunk
};

// -------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until flag == epoch. Returns false (and raises *err) when the budget
// is exhausted, or at once when another thread has raised *err.
__device__ __forceinline__ bool wait_ready(const unsigned* flag, unsigned epoch, int* err,
                                           unsigned long long deadline) {
  if (ld_acquire(flag) == epoch) return true;
  while (true) {
    if (*(volatile int*)err != 0) return false;
    __nanosleep(32);
    if (ld_acquire(flag) == epoch) return true;
    if (globaltimer() > deadline) {
      atomicExch(err, 1);
      return false;
    }
  }
}

// ------------------------------------------------------------ factor
// Lane = row. Chunk rows never depend on each other (same level).
__global__ void __launch_bounds__(256)
k_ilu_factor(const int* __restrict__ rowptr, const int* __restrict__ col,
             const int* __restrict__ diagpos, double* F, const int* __restrict__ order,
             const int* __restrict__ chunk, int nchunk, unsigned* flags, unsigned epoch,
             int* ticket, int* err) {
  const unsigned long long deadline = globaltimer() + kWaitBudgetNs;
  const int lane = threadIdx.x & 31;
  while (true) {
    int t = 0;
    if (lane == 0) t = atomicAdd(ticket, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= nchunk) return;
    const int beg = chunk[t], end = chunk[t + 1];
    if (beg + lane < end) {
      const int i = order[beg + lane];
      const int rb = rowptr[i], re = rowptr[i + 1], di = diagpos[i];
      bool ok = true;
      for (int p = rb; p < di; ++p) {
        const int k = col[p];
        if (ok) ok = wait_ready(flags + k, epoch, err, deadline);
        const double ukk = __ldcg(F + diagpos[k]);
        const double lik = F[p] / ukk;
        F[p] = lik;
        int ptr = p + 1;
        const int ke = rowptr[k + 1];
        for (int q = diagpos[k] + 1; q < ke; ++q) {
          const int j = col[q];
          while (ptr < re && col[ptr] < j) ++ptr;
          if (ptr < re && col[ptr] == j) F[ptr] -= lik * __ldcg(F + q);
        }
      }
      const double d = F[di];
      if (!(d != 0.0) || !isfinite(d)) atomicExch(err, 2);
      __threadfence();
      st_release(flags + i, epoch);
    }
  }
}

__global__ void k_cast_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __double2float_rn(a[i]);
}

// ------------------------------------------------------------- apply
// Lane = (row slot, column): RPW = 32 / SP rows per chunk, SP = pow2 >= s.
// FWD: Z_i = X_i - sum_{k<i} L_ik Z_k   (unit lower)
// BWD: Z_i = (Z_i - sum_{j>i} U_ij Z_j) / U_ii   (in place)
template <typename VT, bool FWD>
__global__ void __launch_bounds__(256)
k_ilu_sweep(int s, int sp_log2, const int* __restrict__ rowptr, const int* __restrict__ col,
            const int* __restrict__ diagpos, const VT* __restrict__ F, const int* __restrict__ order,
            const int* __restrict__ chunk, int nchunk, const VT* X, VT* Z, unsigned* flags,
            unsigned epoch, int* ticket, int* err) {
  const unsigned long long deadline = globaltimer() + kWaitBudgetNs;
  const int lane = threadIdx.x & 31;
  const int slot = lane >> sp_log2;
  const int k = lane & ((1 << sp_log2) - 1);
  while (true) {
    int t = 0;
    if (lane == 0) t = atomicAdd(ticket, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= nchunk) return;
    const int beg = chunk[t], end = chunk[t + 1];
    const bool row_ok = beg + slot < end;
    const bool act = row_ok && k < s;
    int i = 0;
    if (row_ok) {
      i = order[beg + slot];
      const int di = diagpos[i];
      bool ok = true;
      VT acc;
      if (FWD) {
        acc = act ? X[(int64_t)i * s + k] : VT(0);
        for (int p = rowptr[i]; p < di; ++p) {
          const int c = col[p];
          if (ok) ok = wait_ready(flags + c, epoch, err, deadline);
          if (act) acc -= F[p] * __ldcg(Z + (int64_t)c * s + k);
        }
      } else {
        acc = act ? __ldcg(Z + (int64_t)i * s + k) : VT(0);
        const int re = rowptr[i + 1];
        for (int p = di + 1; p < re; ++p) {
          const int c = col[p];
          if (ok) ok = wait_ready(flags + c, epoch, err, deadline);
          if (act) acc -= F[p] * __ldcg(Z + (int64_t)c * s + k);
        }
        acc /= F[di];
      }
      if (act) Z[(int64_t)i * s + k] = acc;
      __threadfence();
    }
    __syncwarp();
    if (row_ok && k == 0) st_release(flags + i, epoch);
  }
}

// ------------------------------------------------------------ host side
static void levels(const pint_op op, bool forward, std::vector<int>& order,
                   std::vector<int>& lvlptr) {
  const int64_t n = op->n;
  const auto& rp = op->h_rowptr;
  const auto& ci = op->h_colind;
  std::vector<int> lv(n, 0);
  int maxl = 0;
  if (forward) {
    for (int64_t i = 0; i < n; ++i) {
      int l = 0;
      for (int p = rp[i]; p < rp[i + 1]; ++p)
        if (ci[p] < i) l = std::max(l, lv[ci[p]] + 1);
      lv[i] = l;
      maxl = std::max(maxl, l);
    }
  } else {
    for (int64_t i = n - 1; i >= 0; --i) {
      int l = 0;
      for (int p = rp[i]; p < rp[i + 1]; ++p)
        if (ci[p] > i) l = std::max(l, lv[ci[p]] + 1);
      lv[i] = l;
      maxl = std::max(maxl, l);
    }
  }
  lvlptr.assign(maxl + 2, 0);
  for (int64_t i = 0; i < n; ++i) lvlptr[lv[i] + 1]++;
  for (int l = 0; l <= maxl; ++l) lvlptr[l + 1] += lvlptr[l];
  order.resize(n);
  std::vector<int> pos(lvlptr.begin(), lvlptr.end() - 1);
  for (int64_t i = 0; i < n; ++i) order[pos[lv[i]]++] = (int)i;
}

static Sched& schedule(pint_op op, bool forward, int rpw) {
  IluState* S = op->ilu;
  auto& cache = forward ? S->sched_f : S->sched_b;
  auto it = cache.find(rpw);
  if (it != cache.end()) return it->second;
  const auto& lp = forward ? S->lvlptr_f : S->lvlptr_b;
  std::vector<int> ch;
  for (size_t l = 0; l + 1 < lp.size(); ++l)
    for (int b = lp[l]; b < lp[l + 1]; b += rpw) ch.push_back(b);
  ch.push_back((int)op->n);
  Sched sc;
  sc.nchunk = (int)ch.size() - 1;
  sc.order = forward ? S->d_order_f : S->d_order_b;
  sc.bytes_chunk = sizeof(int) * ch.size();
  sc.chunk = (int*)dalloc(op->ctx, sc.bytes_chunk);
  PINT_CUDA(cudaMemcpy(sc.chunk, ch.data(), sc.bytes_chunk, cudaMemcpyHostToDevice));
  return cache.emplace(rpw, sc).first->second;
}

static unsigned next_epoch(pint_op op, unsigned& e, unsigned* flags, cudaStream_t st) {
  if (e >= 0xFFFFFF00u) {
    PINT_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned) * op->n, st));
    e = 0;
  }
  return ++e;
}

static void ensure_state(pint_op op) {
  if (op->ilu) return;
  IluState* S = new IluState();
  op->ilu = S;
  pint_ctx ctx = op->ctx;
  levels(op, true, S->order_f, S->lvlptr_f);
  levels(op, false, S->order_b, S->lvlptr_b);
  S->F64 = dalloc_n<double>(ctx, op->nnz);
  S->F32 = dalloc_n<float>(ctx, op->nnz);
  S->flag_f = dalloc_n<unsigned>(ctx, op->n);
  S->flag_b = dalloc_n<unsigned>(ctx, op->n);
  S->ticket = dalloc_n<int>(ctx, 2);
  S->err = dalloc_n<int>(ctx, 2);
  S->d_order_f = dalloc_n<int>(ctx, op->n);
  S->d_order_b = dalloc_n<int>(ctx, op->n);
  PINT_CUDA(cudaMemcpy(S->d_order_f, S->order_f.data(), sizeof(int) * op->n, cudaMemcpyHostToDevice));
  PINT_CUDA(cudaMemcpy(S->d_order_b, S->order_b.data(), sizeof(int) * op->n, cudaMemcpyHostToDevice));
  PINT_CUDA(cudaMemset(S->flag_f, 0, sizeof(unsigned) * op->n));
  PINT_CUDA(cudaMemset(S->flag_b, 0, sizeof(unsigned) * op->n));
  PINT_CUDA(cudaMemset(S->err, 0, 2 * sizeof(int)));
}

static unsigned sweep_grid(pint_op op, int nchunk) {
  const int warps = std::max(1, std::min(nchunk, op->ctx->num_sms * 16));
  return (unsigned)((warps + 7) / 8);
}

void ilu_destroy(pint_op op) {
  IluState* S = op->ilu;
  if (!S) return;
  pint_ctx c = op->ctx;
  for (auto* m : {&S->sched_f, &S->sched_b})
    for (auto& kv : *m) dfree(c, kv.second.chunk, kv.second.bytes_chunk);
  dfree(c, S->F64, sizeof(double) * op->nnz);
  dfree(c, S->F32, sizeof(float) * op->nnz);
  dfree(c, S->flag_f, sizeof(unsigned) * op->n);
  dfree(c, S->flag_b, sizeof(unsigned) * op->n);
  dfree(c, S->ticket, 2 * sizeof(int));
  dfree(c, S->err, 2 * sizeof(int));
  dfree(c, S->d_order_f, sizeof(int) * op->n);
  dfree(c, S->d_order_b, sizeof(int) * op->n);
  delete S;
  op->ilu = nullptr;
}

void ilu_check(pint_op op) {
  IluState* S = op->ilu;
  if (!S) return;
  int e = 0;
  PINT_CUDA(cudaMemcpy(&e, S->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e == 1) throw Error{PINT_ERR_TIMEOUT, "ILU(0) dependency wait exceeded its time budget"};
  if (e == 2) throw Error{PINT_ERR_BREAKDOWN, "ILU(0) zero or non-finite pivot"};
}

void ilu_setup(pint_op op, cudaStream_t st) {
  ensure_state(op);
  IluState* S = op->ilu;
  if (S->factored) return;
  if (!op->j_valid) build_inner(op, st);
  PINT_CUDA(cudaMemcpyAsync(S->F64, op->Jval, sizeof(double) * op->nnz, cudaMemcpyDeviceToDevice, st));
  PINT_CUDA(cudaMemsetAsync(S->err, 0, 2 * sizeof(int), st));
  Sched& sc = schedule(op, true, 32);
  const unsigned ep = next_epoch(op, S->epoch_f, S->flag_f, st);
  PINT_CUDA(cudaMemsetAsync(S->ticket, 0, sizeof(int), st));
  ProfScope ps(op->ctx, PF_ILU, op->nnz * 28.0 + 12.0 * op->n, 2.0 * op->nnz * 3, st);
  k_ilu_factor<<<sweep_grid(op, sc.nchunk), 256, 0, st>>>(op->rowptr, op->colind, op->diagpos,
                                                          S->F64, sc.order, sc.chunk, sc.nchunk,
                                                          S->flag_f, ep, S->ticket, S->err);
  check_launch("k_ilu_factor");
  k_cast_f32<<<grid_for(op->nnz, 256), 256, 0, st>>>(op->nnz, S->F64, S->F32);
  check_launch("k_cast_f32");
  op->ctx->launches += 2;
  PINT_CUDA(cudaStreamSynchronize(st));
  ilu_check(op);
  S->factored = true;
}

template <typename VT>
static void apply_t(pint_op op, const VT* F, const VT* X, VT* Z, cudaStream_t st) {
  IluState* S = op->ilu;
  const int s = op->s;
  int spl = 0;
  while ((1 << spl) < s) ++spl;
  const int rpw = 32 >> spl;
  Sched& f = schedule(op, true, rpw);
  Sched& b = schedule(op, false, rpw);
  const unsigned ef = next_epoch(op, S->epoch_f, S->flag_f, st);
  const unsigned eb = next_epoch(op, S->epoch_b, S->flag_b, st);
  PINT_CUDA(cudaMemsetAsync(S->ticket, 0, 2 * sizeof(int), st));
  ProfScope ps(op->ctx, PF_ILU,
               op->nnz * (sizeof(VT) + 4.0) + 4.0 * (op->n + 1) + 8.0 * op->n + 8.0 * op->n +
                   4.0 * sizeof(VT) * op->n * s,
               2.0 * op->nnz * s, st);
  k_ilu_sweep<VT, true><<<sweep_grid(op, f.nchunk), 256, 0, st>>>(
      s, spl, op->rowptr, op->colind, op->diagpos, F, f.order, f.chunk, f.nchunk, X, Z, S->flag_f,
      ef, S->ticket, S->err);
  check_launch("k_ilu_sweep<fwd>");
  k_ilu_sweep<VT, false><<<sweep_grid(op, b.nchunk), 256, 0, st>>>(
      s, spl, op->rowptr, op->colind, op->diagpos, F, b.order, b.chunk, b.nchunk, Z, Z, S->flag_b,
      eb, S->ticket + 1, S->err);
  check_launch("k_ilu_sweep<bwd>");
  op->ctx->launches += 2;
}

void ilu_apply(pint_op op, int precision, const void* X, void* Z, cudaStream_t st) {
  PINT_REQUIRE(op->ilu && op->ilu->factored, PINT_ERR_INVALID, "ILU(0) not set up");
  if (precision == PINT_FP64)
    apply_t<double>(op, op->ilu->F64, (const double*)X, (double*)Z, st);
  else
    apply_t<float>(op, op->ilu->F32, (const float*)X, (float*)Z, st);
}

}  // namespace pint
