// Batched slab solves: one persistent launch whose thread-block clusters take
// slab-solve jobs from a device queue and solve each job entirely inside the
// cluster, so that many small solves (uneven N and s, each its own operator
// and coupling) share one launch and need no host round trip per Arnoldi step.
//
// Per job the method is the global GMRES slab solve of the unsplit operator
// A(V) = M V A1^T + K V A2^T (Eq. general-system-time-steps; the library's
// PINT_SOLVER_GLOBAL): defect correction with restarts, R = R(Y), global
// GMRES(m) on A(D^-1 V) = R from V = 0 in the Frobenius inner product
// (Givens rotations on the scalar Hessenberg matrix), Y <- Y - D^-1 Z with D
// the diagonal of J = alpha M + beta K (right Jacobi preconditioning),
// stopping per column on ||R_k|| <= tol ||F_k||.
//
// A cluster of C CTAs (C = 1..16) shares one job: CTA q owns rows
// [q N / C, (q+1) N / C) of every N x s block. Reductions go warp -> CTA ->
// cluster: each CTA writes its partial sums to its own shared memory, the
// cluster barrier (release/acquire at cluster scope) publishes them, and every
// CTA adds the C partials in rank order through distributed shared memory, so
// all CTAs hold bitwise the same sums and take the same branches. The small
// least-squares state (Hessenberg matrix, rotations) is kept and updated
// redundantly by every CTA. Operand rows owned by another CTA are read with
// L2-only loads after a cluster barrier.
//
// Float64 arithmetic is the scarce resource on this GPU (about 1/64 of the
// float32 rate), so the kernel counts float64 instructions rather than bytes:
// the Jacobi-scaled values of K and the row factors of M D^-1 are formed once
// per job; the s x s products skip the zero entries of A1 and A2 (lists built
// per job); warp sums of several values use a transposing butterfly (6 adds
// for 4 values instead of 20); normalisations multiply by a reciprocal. With
// one CTA per job the Arnoldi vectors are orthogonalised by modified
// Gram-Schmidt (one product and one update per basis vector, half the
// float64 work of two classical passes, and a CTA barrier per product); with
// a cluster per job by two classical Gram-Schmidt passes (three reductions
// per step, each a cluster barrier). Reductions run in a fixed order for a
// given C, so a job's result does not depend on the other jobs of the batch.
#include "internal.h"

#include <cooperative_groups.h>

#include <algorithm>
#include <chrono>
#include <cmath>

namespace cg = cooperative_groups;

namespace pint {

struct BatchJob {
  int64_t n, nnz;
  int s;
  int orig;                 // the caller's index of this job (its output slot)
  const int* rowptr;        // CSR of K (device)
  const int* colind;
  const double* Kval;
  const double* Mdiag;      // nullptr: M = I
  const double* Jinv;       // 1 / diag(J), J = alpha M + beta K (ones: no preconditioner)
  const double* cpl;        // A1 then A2, row-major s x s each (device)
  const double* B;          // N x s or nullptr
  const double* B0;         // N x s or nullptr
  double* Y;                // N x s, in: initial guess, out: solution
};

struct BatchOut {
  int status, outer, inner, cycles;
  long long flops;          // algorithmic float64 operations of the job (FMA = 2)
  double relres[kMaxS];
};

constexpr int kBatchThreadsMax = 512;  // CTA widths 128, 256, 512 (a template parameter)
constexpr int kRedSlot = 32;          // values per cluster reduction (m + 1 <= 31, s <= 16)

// Sum over the warp of NV = 2^p values per lane with NV - 1 + 5 - p adds:
// at each halving step a lane keeps half of its values, sends the other half
// to its partner and adds what it receives; plain butterfly steps follow.
// Lane l ends with the total of value l >> (5 - p).
template <int NV>
__device__ __forceinline__ double warp_sum_multi(double (&a)[NV]) {
  const int lane = threadIdx.x & 31;
  int o = 16;
#pragma unroll
  for (int c = NV; c > 1; c >>= 1) {
    const bool up = lane & o;
#pragma unroll
    for (int t = 0; t < c / 2; ++t) {
      const double send = up ? a[t] : a[t + c / 2];
      const double keep = up ? a[t + c / 2] : a[t];
      a[t] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    o >>= 1;
  }
  double v = a[0];
#pragma unroll
  for (int q = 0; q < 5; ++q)
    if ((16 >> q) <= o) v += __shfl_xor_sync(0xffffffffu, v, 16 >> q);
  return v;
}

// Nonzero entries of A1 and A2 by row (built per job): row i of A1 is
// k[off[i] .. off[i+1]) with values v[...]; A2 likewise after A1.
struct CplLists {
  int off1[kMaxS + 1], off2[kMaxS + 1];
  int k[2 * kMaxS * kMaxS];
  double v[2 * kMaxS * kMaxS];
};

// Rows [r0, r1) of out = d .* (X A1^T) + (K X - B) A2^T - B0 for one job with
// s = S. PRE: the preconditioned Krylov operator (K values and d already
// scaled by D^-1, no B, B0); else the residual (K values, d = diag(M)). X may
// hold rows written by other CTAs of the cluster: read at L2. The s x s
// products run over the nonzero lists, through a per-thread staging area xs
// (2 S doubles per thread, stride blockDim.x), in increasing column order.
template <int S, bool PRE>
__device__ __noinline__ void coupled_rows(int64_t n, int64_t r0, int64_t r1,
                                          const int* __restrict__ rowptr,
                                          const int* __restrict__ colind,
                                          const double* __restrict__ Kv,
                                          const double* __restrict__ dg, const CplLists& L,
                                          const double* __restrict__ X,
                                          const double* __restrict__ B,
                                          const double* __restrict__ B0,
                                          double* __restrict__ out, double* xs) {
  const int T = blockDim.x;
  double* xt = xs + threadIdx.x;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += T) {
    double ky[S];
#pragma unroll
    for (int k = 0; k < S; ++k) ky[k] = 0.0;
    const int p1 = rowptr[r + 1];
    for (int p = rowptr[r]; p < p1; ++p) {
      const double v = Kv[p];
      if (!PINT_INDEX_OK(colind[p], n, 3)) continue;
      const double* xc = X + (int64_t)colind[p] * S;
#pragma unroll
      for (int k = 0; k < S; ++k) ky[k] = fma(v, __ldcg(xc + k), ky[k]);
    }
#pragma unroll
    for (int k = 0; k < S; ++k) {
      xt[k * T] = __ldcg(X + r * S + k);
      xt[(S + k) * T] = (!PRE && B) ? ky[k] - B[r * S + k] : ky[k];
    }
    const double d = dg ? dg[r] : 1.0;
    for (int i = 0; i < S; ++i) {
      double m1 = 0.0, m2 = 0.0;
      for (int q = L.off1[i]; q < L.off1[i + 1]; ++q) m1 = fma(L.v[q], xt[L.k[q] * T], m1);
      for (int q = L.off2[i]; q < L.off2[i + 1]; ++q)
        m2 = fma(L.v[q], xt[(S + L.k[q]) * T], m2);
      double o = fma(d, m1, m2);
      if (!PRE && B0) o -= B0[r * S + i];
      out[r * S + i] = o;
    }
  }
}

template <bool PRE>
__device__ __forceinline__ void coupled(int s, int64_t n, int64_t r0, int64_t r1,
                                        const int* rowptr,
                                        const int* colind, const double* Kv, const double* dg,
                                        const CplLists& L, const double* X, const double* B,
                                        const double* B0, double* out, double* xs) {
  switch (s) {
#define PINT_CASE(SS) \
  case SS: coupled_rows<SS, PRE>(n, r0, r1, rowptr, colind, Kv, dg, L, X, B, B0, out, xs); break;
    PINT_CASE(1) PINT_CASE(2) PINT_CASE(3) PINT_CASE(4) PINT_CASE(5) PINT_CASE(6)
    PINT_CASE(7) PINT_CASE(8) PINT_CASE(9) PINT_CASE(10) PINT_CASE(11) PINT_CASE(12)
    PINT_CASE(13) PINT_CASE(14) PINT_CASE(15) PINT_CASE(16)
#undef PINT_CASE
    default: break;
  }
}

// Squared column norms of rows [r0, r1) of X (N x S): warp partials of
// column k into red2[k * NW + warp].
template <int S, int NW>
__device__ __noinline__ void colsq_rows(int64_t r0, int64_t r1, const double* X, double* red2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double acc[S];
#pragma unroll
  for (int k = 0; k < S; ++k) acc[k] = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x)
#pragma unroll
    for (int k = 0; k < S; ++k) acc[k] = fma(X[r * S + k], X[r * S + k], acc[k]);
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) red2[k * NW + warp] = v;
  }
}

template <int NW>
__device__ __forceinline__ void colsq(int s, int64_t r0, int64_t r1, const double* X,
                                      double* red2) {
  switch (s) {
#define PINT_CASE(SS) \
  case SS: colsq_rows<SS, NW>(r0, r1, X, red2); break;
    PINT_CASE(1) PINT_CASE(2) PINT_CASE(3) PINT_CASE(4) PINT_CASE(5) PINT_CASE(6)
    PINT_CASE(7) PINT_CASE(8) PINT_CASE(9) PINT_CASE(10) PINT_CASE(11) PINT_CASE(12)
    PINT_CASE(13) PINT_CASE(14) PINT_CASE(15) PINT_CASE(16)
#undef PINT_CASE
    default: break;
  }
}

// Cluster sum of nv <= kRedSlot values: the warp partials of value v are in
// red2[v * NW + w] (NW warps). Every CTA of the cluster ends with the same sums
// in res[0..nv): CTA partials (warps in order) go to this CTA's slot, the
// cluster barrier publishes them, and each CTA adds the slots of ranks
// 0..C-1 in order. Callers alternate between two slots, so a slot is
// rewritten only after the next barrier has shown that every CTA is done
// reading it. With C = 1 the cluster barrier is a CTA barrier.
template <int NW>
__device__ __forceinline__ void cluster_reduce(cg::cluster_group& cl, int C, int nv,
                                               const double* red2, double* slot, double* res) {
  __syncthreads();
  const int t = threadIdx.x;
  if (nv == 1) {                  // one value: a tree over the warp partials
    if (t < 32) {
      double a = t < NW ? red2[t] : 0.0;
      a = warp_sum(a);
      if (t == 0) {
        if (C == 1) res[0] = a;
        else slot[0] = a;
      }
    }
  } else if (t < nv) {
    double a = 0.0;
    for (int w = 0; w < NW; ++w) a += red2[t * NW + w];
    if (C == 1) res[t] = a;
    else slot[t] = a;
  }
  if (C == 1) {
    __syncthreads();
    return;
  }
  cl.sync();
  if (t < nv) {
    double a = 0.0;
    for (int q = 0; q < C; ++q) a += cl.map_shared_rank(slot, q)[t];
    res[t] = a;
  }
  __syncthreads();
}

// Frobenius products of NV consecutive basis blocks P_u = P + u ns with W over
// the elements [e0, e1) of this CTA; warp partials of product i0 + u go to
// red2[(i0 + u) * NW + warp].
template <int NV, int NW>
__device__ __forceinline__ void dots_chunk(const double* P, int64_t ns, const double* W,
                                           int64_t e0, int64_t e1, int i0, double* red2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double a[NV];
#pragma unroll
  for (int u = 0; u < NV; ++u) a[u] = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const double w = W[e];
#pragma unroll
    for (int u = 0; u < NV; ++u) a[u] = fma(P[u * ns + e], w, a[u]);
  }
  const double v = warp_sum_multi<NV>(a);
  constexpr int per = 32 / NV;
  if (lane % per == 0) red2[(i0 + lane / per) * NW + warp] = v;
}

// One modified Gram-Schmidt sweep over the elements [e0, e1) of this CTA:
// W <- W - h Vi, returning this thread's partial of <Vn, W> for the updated W
// (Vn != nullptr) or of ||W||^2. Four elements per round with all loads
// issued before the stores (the three blocks never overlap), so a thread
// keeps twelve loads in flight instead of three.
__device__ __forceinline__ double mgs_sweep(const double* __restrict__ Vi,
                                            const double* __restrict__ Vn,
                                            double* __restrict__ W, double h, int64_t e0,
                                            int64_t e1) {
  const int T = blockDim.x;
  double a = 0.0;
  int64_t e = e0 + threadIdx.x;
  for (; e + 3 * (int64_t)T < e1; e += 4 * (int64_t)T) {
    double v[4], w[4], q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      v[u] = Vi[e + u * T];
      w[u] = W[e + u * T];
      q[u] = Vn ? Vn[e + u * T] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      w[u] = fma(-h, v[u], w[u]);
      W[e + u * T] = w[u];
      a = fma(Vn ? q[u] : w[u], w[u], a);
    }
  }
  for (; e < e1; e += T) {
    const double w = fma(-h, Vi[e], W[e]);
    W[e] = w;
    a = fma(Vn ? Vn[e] : w, w, a);
  }
  return a;
}

// Products <V_i, W> for i = 0..j in chunks of 8, 4, 2, 1.
template <int NW>
__device__ __forceinline__ void dots_all(const double* V, int64_t ns, const double* W, int j,
                                         int64_t e0, int64_t e1, double* red2) {
  int i0 = 0, left = j + 1;
  while (left >= 8) {
    dots_chunk<8, NW>(V + (size_t)i0 * ns, ns, W, e0, e1, i0, red2);
    i0 += 8;
    left -= 8;
  }
  if (left >= 4) {
    dots_chunk<4, NW>(V + (size_t)i0 * ns, ns, W, e0, e1, i0, red2);
    i0 += 4;
    left -= 4;
  }
  if (left >= 2) {
    dots_chunk<2, NW>(V + (size_t)i0 * ns, ns, W, e0, e1, i0, red2);
    i0 += 2;
    left -= 2;
  }
  if (left >= 1) dots_chunk<1, NW>(V + (size_t)i0 * ns, ns, W, e0, e1, i0, red2);
}

// Dynamic shared memory of k_slab_queue (doubles) for restart length m,
// largest block width smax and nt threads: Hessenberg (m+1) x m, g, cs, sn,
// y, h (m+1 each), warp partials kRedSlot x warps, two cluster slots and the
// reduced values (kRedSlot each), ||F_k||, ||R_k||, scalars, the coupling
// staging area (2 smax per thread).
__host__ __device__ inline size_t batch_smem_doubles(int m, int smax, int nt) {
  return (size_t)(m + 1) * m + 5 * (size_t)(m + 1) + (size_t)kRedSlot * (nt / 32) +
         3 * kRedSlot + 2 * kMaxS + 8 + 2 * (size_t)smax * nt;
}

// Per-cluster workspace of one job (doubles): m + 1 basis blocks, R, Z (N s
// each), the Jacobi-scaled values of K (nnz) and the row factors of M D^-1 (N).
__host__ __device__ inline int64_t batch_work_doubles(int m, int64_t n, int s, int64_t nnz) {
  return (int64_t)(m + 3) * n * s + nnz + n;
}

// Persistent batched slab solver: each cluster takes jobs from *queue until
// the queue is empty. Every branch that brackets a barrier depends only on
// values that all CTAs of the cluster hold identically (cluster sums, the
// redundantly updated least-squares state, iteration counters).
template <int NT>
__global__ void __launch_bounds__(NT, kBatchThreadsMax / NT)
k_slab_queue(int njobs, const BatchJob* __restrict__ jobs, int m, double tol, int max_outer,
             int max_inner, double* __restrict__ work, int64_t work_stride,
             int* __restrict__ queue, BatchOut* __restrict__ outs) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const bool mgs = C == 1;
  extern __shared__ __align__(16) double sm[];
  double* H = sm;                                    // (m+1) x m, pitch m
  double* g = H + (size_t)(m + 1) * m;
  double* cs = g + (m + 1);
  double* sn = cs + (m + 1);
  double* y = sn + (m + 1);
  double* hs = y + (m + 1);
  double* red2 = hs + (m + 1);                       // kRedSlot x warps
  constexpr int NW = NT / 32;
  double* slots = red2 + (size_t)kRedSlot * NW;     // 2 x kRedSlot
  double* res = slots + 2 * kRedSlot;                // kRedSlot
  double* fn = res + kRedSlot;                       // kMaxS
  double* rn = fn + kMaxS;                           // kMaxS
  double* misc = rn + kMaxS;                         // 8 scalars
  double* xs = misc + 8;                             // 2 smax x threads
  __shared__ CplLists L;
  __shared__ BatchJob J;                             // the current job (read on use)
  __shared__ int job_sh;
  const int tid = threadIdx.x, T = blockDim.x, warp = tid >> 5, lane = tid & 31;
  double* ws = work + (int64_t)(blockIdx.x / C) * work_stride;
  int buf = 0;                                       // cluster slot in use
#define PINT_REDUCE(NV)                                                 \
  do {                                                                  \
    cluster_reduce<NW>(cl, C, (NV), red2, slots + buf * kRedSlot, res); \
    buf ^= 1;                                                           \
  } while (0)
#define PINT_SYNC_ALL() \
  do {                  \
    if (C > 1)          \
      cl.sync();        \
    else                \
      __syncthreads();  \
  } while (0)
  while (true) {
    if (rank == 0 && tid == 0) job_sh = atomicAdd(queue, 1);
    cl.sync();
    const int jb = *cl.map_shared_rank(&job_sh, 0);
    if (jb >= njobs) {
      cl.sync();               // rank 0's shared memory stays until all have read it
      return;
    }
    if (tid == 0) J = jobs[jb];
    __syncthreads();
    const int s = J.s;
    const int64_t n = J.n, ns = n * s;
    const int64_t r0 = n * rank / C, r1 = n * (rank + 1) / C;
    const int64_t e0 = r0 * s, e1 = r1 * s;
    double* V = ws;                                  // (m+1) blocks of N x s
    double* R = V + (size_t)(m + 1) * ns;
    double* Z = R + ns;
    double* Kt = Z + ns;                             // nnz
    double* dm = Kt + J.nnz;                         // N
    if (tid == 0) {                                  // nonzero lists of A1, A2
      int q = 0;
      for (int i = 0; i < s; ++i) {
        L.off1[i] = q;
        for (int k = 0; k < s; ++k)
          if (J.cpl[i * s + k] != 0.0) {
            L.k[q] = k;
            L.v[q++] = J.cpl[i * s + k];
          }
      }
      L.off1[s] = q;
      for (int i = 0; i < s; ++i) {
        L.off2[i] = q;
        for (int k = 0; k < s; ++k)
          if (J.cpl[s * s + i * s + k] != 0.0) {
            L.k[q] = k;
            L.v[q++] = J.cpl[s * s + i * s + k];
          }
      }
      L.off2[s] = q;
    }
    for (int64_t p = J.rowptr[r0] + tid; p < J.rowptr[r1]; p += T)
      Kt[p] = J.Kval[p] * J.Jinv[J.colind[p]];
    for (int64_t r = r0 + tid; r < r1; r += T) dm[r] = (J.Mdiag ? J.Mdiag[r] : 1.0) * J.Jinv[r];
    for (int64_t e = e0 + tid; e < e1; e += T) Z[e] = 0.0;
    cl.sync();
    // ||F_k|| from the residual of Y = 0
    coupled<false>(s, n, r0, r1, J.rowptr, J.colind, J.Kval, J.Mdiag, L, Z, J.B, J.B0, R, xs);
    colsq<NW>(s, r0, r1, R, red2);
    PINT_REDUCE(s);
    if (tid < s) fn[tid] = sqrt(res[tid]);
    __syncthreads();
    double target = 0.0;
    for (int k = 0; k < s; ++k) {
      const double thr = fn[k] > 0.0 ? tol * fn[k] : tol;
      target = k == 0 ? thr : fmin(target, thr);
    }
    int status = PINT_ERR_NOT_CONVERGED, outer = 0, inner = 0, cycles = 0;
    // algorithmic float64 operation count (FMA = 2): residual and Krylov
    // operator per application, per-step orthogonalisation, per-cycle update
    const long long nA = L.off2[s];                  // nonzeros of A1 and A2
    const long long c_pre = 2LL * J.nnz * s + 2LL * n * nA + 2LL * ns;
    const long long c_res = c_pre + (J.B ? ns : 0) + (J.B0 ? ns : 0);
    long long flops = (long long)J.nnz + n + c_res + 2LL * ns;
    for (outer = 0; outer <= max_outer; ++outer) {
      flops += c_res + 2LL * ns;
      PINT_SYNC_ALL();                               // Y rows of every CTA updated
      coupled<false>(s, n, r0, r1, J.rowptr, J.colind, J.Kval, J.Mdiag, L, J.Y, J.B, J.B0, R, xs);
      colsq<NW>(s, r0, r1, R, red2);
      PINT_REDUCE(s);
      if (tid < s) rn[tid] = sqrt(res[tid]);
      __syncthreads();
      bool done = true, bad = false;
      double beta = 0.0;
      for (int k = 0; k < s; ++k) {
        if (!isfinite(rn[k])) bad = true;
        if (!(rn[k] <= (fn[k] > 0.0 ? tol * fn[k] : tol))) done = false;
        beta = fma(rn[k], rn[k], beta);
      }
      beta = sqrt(beta);
      if (bad) {
        status = PINT_ERR_BREAKDOWN;
        break;
      }
      if (done) {
        status = PINT_OK;
        break;
      }
      if (outer == max_outer || inner >= max_inner) break;
      cycles += 1;
      flops += ns;
      // V_0 = R / ||R||_F, least-squares right-hand side beta e_1
      const double ib = 1.0 / beta;
      for (int64_t e = e0 + tid; e < e1; e += T) V[e] = R[e] * ib;
      if (tid == 0) {
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        for (int i = 0; i < (m + 1) * m; ++i) H[i] = 0.0;
        g[0] = beta;
      }
      int j = 0;
      for (j = 0; j < m; ++j) {
        PINT_SYNC_ALL();                             // V_j rows of every CTA written
        const double* Vj = V + (size_t)j * ns;
        double* W = V + (size_t)(j + 1) * ns;
        coupled<true>(s, n, r0, r1, J.rowptr, J.colind, Kt, dm, L, Vj, nullptr, nullptr, W, xs);
        __syncthreads();
        double nw2 = 0.0;
        if (mgs) {
          // modified Gram-Schmidt: h_i = <V_i, W>, W <- W - h_i V_i in turn;
          // each update sweep also forms the next product (or ||W||^2)
          double a = 0.0;
          for (int64_t e = e0 + tid; e < e1; e += T) a = fma(V[e], W[e], a);
          for (int i = 0; i <= j; ++i) {
            a = warp_sum(a);
            if (lane == 0) red2[warp] = a;
            PINT_REDUCE(1);
            const double h = res[0];
            if (tid == 0) H[i * m + j] = h;
            const double* Vi = V + (size_t)i * ns;
            a = mgs_sweep(Vi, i < j ? Vi + ns : nullptr, W, h, e0, e1);
          }
          a = warp_sum(a);
          if (lane == 0) red2[warp] = a;
          PINT_REDUCE(1);
          nw2 = res[0];
        } else {
          // two classical Gram-Schmidt passes; the second update sweep also
          // forms ||W||^2
          double a = 0.0;
          for (int pass = 0; pass < 2; ++pass) {
            dots_all<NW>(V, ns, W, j, e0, e1, red2);
            PINT_REDUCE(j + 1);
            if (tid <= j) {
              hs[tid] = res[tid];
              H[tid * m + j] += res[tid];
            }
            __syncthreads();
            for (int64_t e = e0 + tid; e < e1; e += T) {
              double w = W[e];
              for (int i = 0; i <= j; ++i) w = fma(-hs[i], V[(size_t)i * ns + e], w);
              W[e] = w;
              if (pass == 1) a = fma(w, w, a);
            }
          }
          a = warp_sum(a);
          if (lane == 0) red2[warp] = a;
          PINT_REDUCE(1);
          nw2 = res[0];
        }
        // V_{j+1} = W / ||W||_F and the Givens-reduced Hessenberg column
        const double nw = sqrt(nw2);
        const double iw = nw > 0.0 ? 1.0 / nw : 0.0;
        for (int64_t e = e0 + tid; e < e1; e += T) W[e] *= iw;
        if (tid == 0) {
          H[(j + 1) * m + j] = nw;
          for (int i = 0; i < j; ++i) {
            const double p = H[i * m + j], q = H[(i + 1) * m + j];
            H[i * m + j] = fma(cs[i], p, sn[i] * q);
            H[(i + 1) * m + j] = fma(-sn[i], p, cs[i] * q);
          }
          const double p = H[j * m + j], q = H[(j + 1) * m + j];
          const double r = hypot(p, q);
          const double ir = r > 0.0 ? 1.0 / r : 0.0;
          cs[j] = r > 0.0 ? p * ir : 1.0;
          sn[j] = q * ir;
          H[j * m + j] = r;
          H[(j + 1) * m + j] = 0.0;
          g[j + 1] = -sn[j] * g[j];
          g[j] = cs[j] * g[j];
          misc[0] = fabs(g[j + 1]);
        }
        __syncthreads();
        inner += 1;
        flops += c_pre + (mgs ? 4LL : 8LL) * (j + 1) * ns + 3LL * ns;
        const double est = misc[0];
        if (!isfinite(est)) {
          status = PINT_ERR_BREAKDOWN;
          break;
        }
        if (est <= target || inner >= max_inner) {
          j += 1;
          break;
        }
      }
      if (status == PINT_ERR_BREAKDOWN) break;
      const int kd = min(j, m);
      if (tid == 0) {                                // back substitution
        for (int i = kd - 1; i >= 0; --i) {
          double t = g[i];
          for (int c = i + 1; c < kd; ++c) t = fma(-H[i * m + c], y[c], t);
          const double d = H[i * m + i];
          y[i] = d != 0.0 ? t / d : 0.0;
        }
      }
      __syncthreads();
      flops += 2LL * kd * ns + 2LL * ns;
      // Y <- Y - D^-1 sum_i y_i V_i on this CTA's rows
      for (int64_t r = r0 + tid; r < r1; r += T) {
        const double jr = J.Jinv[r];
        for (int k = 0; k < s; ++k) {
          const int64_t e = r * s + k;
          double acc = 0.0;
          for (int i = 0; i < kd; ++i) acc = fma(y[i], V[(size_t)i * ns + e], acc);
          J.Y[e] = fma(-jr, acc, J.Y[e]);
        }
      }
    }
    if (rank == 0 && tid == 0) {
      BatchOut* o = outs + J.orig;
      o->status = status;
      o->outer = outer;
      o->inner = inner;
      o->cycles = cycles;
      o->flops = flops;
      for (int k = 0; k < kMaxS; ++k)
        o->relres[k] = k < s ? (fn[k] > 0.0 ? rn[k] / fn[k] : rn[k]) : 0.0;
    }
    __syncthreads();
  }
#undef PINT_REDUCE
#undef PINT_SYNC_ALL
}

}  // namespace pint

namespace {

// Cluster size for a batch: double C (from 1, up to 16) while the largest
// job's N s per CTA exceeds the batch's total N s per SM (that job would set
// the launch's finishing time) and the largest job keeps at least 256 rows
// per CTA. Measured on 512 uneven slabs (2-D 32^2-64^2, 3-D 16^3-32^3,
// s = 2..16): C = 1, 2, 4, 8 gave 2.7, 3.4, 4.7, 3.9 x 10^7 time-step DOF/s,
// and this rule takes 4; on 608 copies of one 64 x 64 s = 4 slab it takes 1.
int auto_cluster(int num_sms, int njobs, const pint_batch_job* jobs) {
  int64_t total = 0, wmax = 0, nmax = 0;
  for (int i = 0; i < njobs; ++i) {
    const int64_t w = jobs[i].op->n * jobs[i].op->s;
    total += w;
    wmax = std::max(wmax, w);
    nmax = std::max<int64_t>(nmax, jobs[i].op->n);
  }
  const int64_t per_sm = total / std::max(1, num_sms);
  int C = 1;
  while (C < 16 && wmax / C > per_sm && nmax / (2 * C) >= 256) C *= 2;
  return C;
}

// 512 threads (one CTA per SM), 256 for clusters of 16: measured on the 64 x 64
// s = 4 slab, one CTA of 512 beats two of 256 per SM on single-CTA jobs
// (6.2e7 vs 4.8e7 time-step DOF/s for 608 jobs), and 16 x 256 beats 16 x 512
// (4.1 vs 4.2 ms alone, 5.5 vs 8.1 ms for eight jobs, more clusters resident)
int auto_threads(int num_sms, int njobs, int C) {
  (void)num_sms;
  (void)njobs;
  return C >= 16 ? 256 : 512;
}

double batch_now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

cudaLaunchConfig_t batch_config(int grid, int nt, size_t smem, cudaStream_t st,
                                cudaLaunchAttribute* attr, int C) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3((unsigned)nt, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Sets the kernel's launch attributes and returns how many clusters of C
// CTAs can be resident at once. The kernel also declares about 6.5 KB of
// static shared memory, so the dynamic limit is set on every call.
template <int NT>
int slab_queue_clusters(int C, size_t smem, int num_sms, cudaStream_t st) {
  using namespace pint;
  PINT_CUDA(cudaFuncSetAttribute(k_slab_queue<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  if (C > 8)
    PINT_CUDA(cudaFuncSetAttribute(k_slab_queue<NT>,
                                   cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = batch_config(C * num_sms, NT, smem, st, attr, C);
  int ncl = 0;
  PINT_CUDA(cudaOccupancyMaxActiveClusters(&ncl, k_slab_queue<NT>, &cfg));
  return ncl;
}

template <int NT>
void slab_queue_launch(int C, int nclusters, size_t smem, cudaStream_t st, int njobs,
                       const pint::BatchJob* jobs, int m, const pint_opts* o, double* work,
                       int64_t stride, int* queue, pint::BatchOut* outs) {
  using namespace pint;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = batch_config(C * nclusters, NT, smem, st, attr, C);
  PINT_CUDA(cudaLaunchKernelEx(&cfg, k_slab_queue<NT>, njobs, jobs, m, o->tol, o->max_outer,
                               o->max_inner, work, stride, queue, outs));
  check_launch("k_slab_queue");
}

}  // namespace

struct pint_batch_plan_s {
  pint_ctx ctx = nullptr;
  int njobs = 0, m = 0, C = 1, NT = 512, nclusters = 0;
  size_t smem = 0;
  int64_t stride = 0;
  pint_opts o{};
  std::vector<std::pair<void*, size_t>> dev;         // device allocations (budgeted)
  pint::BatchJob* d_jobs = nullptr;
  pint::BatchOut* d_out = nullptr;
  double* d_cpl = nullptr;
  int* d_queue = nullptr;
  double* work = nullptr;
  double* d_ones = nullptr;
  pint::BatchOut* h_out = nullptr;                   // pinned
  cudaStream_t cap = nullptr;                        // private capture stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void* plan_alloc(pint_batch_plan p, size_t b) {
  void* q = pint::dalloc(p->ctx, b);
  p->dev.push_back({q, b});
  return q;
}

void plan_free(pint_batch_plan p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->h_out) cudaFreeHost(p->h_out);
  for (auto& x : p->dev) pint::dfree(p->ctx, x.first, x.second);
  delete p;
}

// Builds the plan: validates the jobs, forms the device descriptors, sizes
// and allocates the workspace, and captures the launch (queue reset + the
// persistent kernel) as a CUDA graph.
void plan_build(pint_batch_plan p, int njobs, const pint_batch_job* jobs, int cluster_ctas,
                int cta_threads, cudaStream_t st) {
  using namespace pint;
  pint_ctx ctx = p->ctx;
  const pint_opts* o = &p->o;
  PINT_REQUIRE(njobs >= 1 && jobs, PINT_ERR_INVALID, "batch: need njobs >= 1 and jobs");
  PINT_REQUIRE(o->precision == PINT_FP64, PINT_ERR_INVALID, "batch: precision must be PINT_FP64");
  PINT_REQUIRE(o->precond == PINT_PC_JACOBI || o->precond == PINT_PC_NONE, PINT_ERR_INVALID,
               "batch: precond must be PINT_PC_JACOBI or PINT_PC_NONE");
  PINT_REQUIRE(o->restart >= 1 && o->restart <= kRedSlot, PINT_ERR_INVALID,
               "batch: restart must be in 1..32");
  PINT_REQUIRE(o->max_outer >= 0 && o->max_inner >= 0 && o->tol >= 0.0, PINT_ERR_INVALID,
               "negative iteration limit or tolerance");
  PINT_REQUIRE(cluster_ctas >= 0 && cluster_ctas <= 16, PINT_ERR_INVALID,
               "cluster_ctas must be 0 (automatic) or 1..16");
  PINT_REQUIRE(cta_threads == 0 || cta_threads == 128 || cta_threads == 256 ||
                   cta_threads == 512,
               PINT_ERR_INVALID, "cta_threads must be 0 (automatic), 128, 256 or 512");
  const int m = o->restart;
  p->njobs = njobs;
  p->m = m;
  int64_t max_work = 1, max_n = 1, ncpl = 0;
  int smax = 1;
  for (int i = 0; i < njobs; ++i) {
    pint_op op = jobs[i].op;
    PINT_REQUIRE(op && op->ctx == ctx, PINT_ERR_INVALID,
                 "batch: every job's operator must belong to ctx");
    PINT_REQUIRE(op->s >= 1, PINT_ERR_INVALID, "coupling not set (pint_set_coupling)");
    PINT_REQUIRE(jobs[i].Y != nullptr, PINT_ERR_INVALID, "batch: job without Y");
    if (!op->j_valid) build_inner(op, st);
    max_work = std::max<int64_t>(max_work, batch_work_doubles(m, op->n, op->s, op->nnz));
    max_n = std::max<int64_t>(max_n, op->n);
    smax = std::max(smax, op->s);
    ncpl += 2 * op->s * op->s;
  }
  p->C = cluster_ctas ? cluster_ctas : auto_cluster(ctx->num_sms, njobs, jobs);
  p->NT = cta_threads ? cta_threads : auto_threads(ctx->num_sms, njobs, p->C);
  p->smem = sizeof(double) * batch_smem_doubles(m, smax, p->NT);
  int ncl = p->NT == 128   ? slab_queue_clusters<128>(p->C, p->smem, ctx->num_sms, st)
            : p->NT == 256 ? slab_queue_clusters<256>(p->C, p->smem, ctx->num_sms, st)
                           : slab_queue_clusters<512>(p->C, p->smem, ctx->num_sms, st);
  PINT_REQUIRE(ncl >= 1, PINT_ERR_INVALID, "batch: a cluster of this size cannot be resident");
  p->nclusters = std::min(ncl, njobs);
  p->stride = ((max_work + 31) / 32) * 32;
  p->d_jobs = static_cast<BatchJob*>(plan_alloc(p, sizeof(BatchJob) * njobs));
  p->d_out = static_cast<BatchOut*>(plan_alloc(p, sizeof(BatchOut) * njobs));
  p->d_cpl = static_cast<double*>(plan_alloc(p, sizeof(double) * ncpl));
  p->d_queue = static_cast<int*>(plan_alloc(p, sizeof(int)));
  p->work = static_cast<double*>(plan_alloc(p, sizeof(double) * (size_t)p->stride * p->nclusters));
  PINT_CUDA(cudaMallocHost(&p->h_out, sizeof(BatchOut) * njobs));
  std::vector<double> ones;
  if (o->precond == PINT_PC_NONE) {
    p->d_ones = static_cast<double*>(plan_alloc(p, sizeof(double) * max_n));
    ones.assign(max_n, 1.0);
    PINT_CUDA(cudaMemcpyAsync(p->d_ones, ones.data(), sizeof(double) * max_n,
                              cudaMemcpyHostToDevice, st));
  }
  // the device queue holds the jobs largest first (N s, then the caller's
  // order): the last jobs a cluster takes are the short ones, which evens out
  // the clusters' finishing times (longest-processing-time-first)
  std::vector<int> order(njobs);
  for (int i = 0; i < njobs; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return jobs[a].op->n * jobs[a].op->s > jobs[b].op->n * jobs[b].op->s;
  });
  std::vector<double> hcpl((size_t)ncpl);
  std::vector<BatchJob> hj(njobs);
  int64_t off = 0;
  for (int q = 0; q < njobs; ++q) {
    const int i = order[q];
    pint_op op = jobs[i].op;
    const int s = op->s;
    for (int a = 0; a < s; ++a)
      for (int b = 0; b < s; ++b) {
        hcpl[off + a * s + b] = op->A1[a * kMaxS + b];
        hcpl[off + s * s + a * s + b] = op->A2[a * kMaxS + b];
      }
    BatchJob& J = hj[q];
    J.n = op->n;
    J.nnz = op->nnz;
    J.s = s;
    J.orig = i;
    J.rowptr = op->rowptr;
    J.colind = op->colind;
    J.Kval = op->Kval;
    J.Mdiag = op->Mdiag;
    J.Jinv = p->d_ones ? p->d_ones : op->Jinvdiag;
    J.cpl = p->d_cpl + off;
    J.B = jobs[i].B;
    J.B0 = jobs[i].B0;
    J.Y = jobs[i].Y;
    off += 2 * s * s;
  }
  PINT_CUDA(cudaMemcpyAsync(p->d_cpl, hcpl.data(), sizeof(double) * ncpl,
                            cudaMemcpyHostToDevice, st));
  PINT_CUDA(cudaMemcpyAsync(p->d_jobs, hj.data(), sizeof(BatchJob) * njobs,
                            cudaMemcpyHostToDevice, st));
  PINT_CUDA(cudaStreamSynchronize(st));             // host staging vectors go out of scope
  // the graph: reset the queue counter, run the persistent kernel
  PINT_CUDA(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
  PINT_CUDA(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(p->d_queue, 0, sizeof(int), p->cap);
  if (p->NT == 128)
    slab_queue_launch<128>(p->C, p->nclusters, p->smem, p->cap, njobs, p->d_jobs, m, o, p->work,
                           p->stride, p->d_queue, p->d_out);
  else if (p->NT == 256)
    slab_queue_launch<256>(p->C, p->nclusters, p->smem, p->cap, njobs, p->d_jobs, m, o, p->work,
                           p->stride, p->d_queue, p->d_out);
  else
    slab_queue_launch<512>(p->C, p->nclusters, p->smem, p->cap, njobs, p->d_jobs, m, o, p->work,
                           p->stride, p->d_queue, p->d_out);
  PINT_CUDA(cudaStreamEndCapture(p->cap, &p->graph));
  PINT_CUDA(cudaGraphInstantiate(&p->exec, p->graph, 0));
}

int plan_run(pint_batch_plan p, pint_stats* stats, cudaStream_t st) {
  using namespace pint;
  const double t0 = batch_now_ms();
  PINT_CUDA(cudaGraphLaunch(p->exec, st));
  check_launch("batch graph");
  p->ctx->launches += 1;
  PINT_CUDA(cudaMemcpyAsync(p->h_out, p->d_out, sizeof(BatchOut) * p->njobs,
                            cudaMemcpyDeviceToHost, st));
  PINT_CUDA(cudaStreamSynchronize(st));
  const double t1 = batch_now_ms();
  int rc = PINT_OK;
  for (int i = 0; i < p->njobs; ++i) {
    const BatchOut& h = p->h_out[i];
    if (stats) {
      pint_stats& S = stats[i];
      S = pint_stats{};
      S.status = h.status;
      S.outer_its = h.outer;
      S.inner_its = h.inner;
      S.restarts = h.cycles;
      S.kernel_launches = 1;
      S.solve_ms = t1 - t0;
      S.flops = (double)h.flops;
      for (int k = 0; k < kMaxS; ++k) S.col_relres[k] = h.relres[k];
    }
    if (h.status == PINT_ERR_BREAKDOWN)
      rc = PINT_ERR_BREAKDOWN;
    else if (h.status != PINT_OK && rc == PINT_OK)
      rc = h.status;
  }
  if (rc == PINT_ERR_BREAKDOWN) p->ctx->err = "batch: non-finite residual in a job";
  else if (rc != PINT_OK) p->ctx->err = "batch: a job did not converge";
  return rc;
}

template <typename Fn>
int batch_guard(pint_ctx ctx, Fn&& fn) {
  if (!ctx) return PINT_ERR_INVALID;
  try {
    PINT_CUDA(cudaSetDevice(ctx->device));
    return fn();
  } catch (const pint::Error& e) {
    ctx->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    ctx->err = "host allocation failed";
    return PINT_ERR_NOMEM;
  }
}

}  // namespace

extern "C" int pint_batch_plan_create(pint_ctx ctx, int njobs, const pint_batch_job* jobs,
                                      const pint_opts* opts, int cluster_ctas, int cta_threads,
                                      pint_batch_plan* plan, void* stream) {
  if (plan) *plan = nullptr;
  return batch_guard(ctx, [&] {
    PINT_REQUIRE(plan && opts, PINT_ERR_INVALID, "batch: need opts and a plan pointer");
    auto* p = new pint_batch_plan_s;
    p->ctx = ctx;
    p->o = *opts;
    try {
      plan_build(p, njobs, jobs, cluster_ctas, cta_threads, static_cast<cudaStream_t>(stream));
    } catch (...) {
      plan_free(p);
      throw;
    }
    *plan = p;
    return PINT_OK;
  });
}

extern "C" int pint_batch_plan_run(pint_batch_plan plan, pint_stats* stats, void* stream) {
  if (!plan) return PINT_ERR_INVALID;
  return batch_guard(plan->ctx,
                     [&] { return plan_run(plan, stats, static_cast<cudaStream_t>(stream)); });
}

extern "C" int pint_batch_plan_shape(pint_batch_plan plan, int* cluster_ctas, int* cta_threads,
                                     int* resident_clusters) {
  if (!plan) return PINT_ERR_INVALID;
  if (cluster_ctas) *cluster_ctas = plan->C;
  if (cta_threads) *cta_threads = plan->NT;
  if (resident_clusters) *resident_clusters = plan->nclusters;
  return PINT_OK;
}

extern "C" int pint_batch_plan_destroy(pint_batch_plan plan) {
  if (!plan) return PINT_ERR_INVALID;
  cudaSetDevice(plan->ctx->device);
  cudaDeviceSynchronize();
  plan_free(plan);
  return PINT_OK;
}

extern "C" int pint_solve_batch(pint_ctx ctx, int njobs, const pint_batch_job* jobs,
                                const pint_opts* o, int cluster_ctas, int cta_threads,
                                pint_stats* stats, void* stream) {
  pint_batch_plan plan = nullptr;
  int rc = pint_batch_plan_create(ctx, njobs, jobs, o, cluster_ctas, cta_threads, &plan, stream);
  if (rc != PINT_OK) return rc;
  rc = pint_batch_plan_run(plan, stats, stream);
  const std::string err = ctx->err;
  pint_batch_plan_destroy(plan);
  ctx->err = err;
  return rc;
}

// Cluster size pint_solve_batch picks for cluster_ctas = 0 (exposed for the
// tuner and the tests).
extern "C" int pint_batch_auto_cluster(pint_ctx ctx, int njobs, const pint_batch_job* jobs) {
  if (!ctx || njobs < 1 || !jobs) return 0;
  for (int i = 0; i < njobs; ++i)
    if (!jobs[i].op || jobs[i].op->s < 1) return 0;
  return auto_cluster(ctx->num_sms, njobs, jobs);
}

// CTA width pint_solve_batch picks for cta_threads = 0.
extern "C" int pint_batch_auto_threads(pint_ctx ctx, int njobs, int cluster_ctas) {
  if (!ctx || njobs < 1 || cluster_ctas < 1) return 0;
  return auto_threads(ctx->num_sms, njobs, cluster_ctas);
}

namespace pint {
void bounds_take_batch(unsigned long long* out) { pint_bounds_take(out); }
}  // namespace pint
