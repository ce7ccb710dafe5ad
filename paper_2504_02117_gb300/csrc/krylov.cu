// Block Krylov inner solve and the outer defect correction.
//
// The matrix equation (alpha M + beta K) Y = RHS of Eq. matrix-fixed-point-
// equation is solved for all s columns at once by block GMRES(m) with right
// preconditioning (the paper uses DUNE-ISTL block Krylov solvers, Sec. 4; it is
// silent on orthogonalisation). Per Arnoldi step:
//   W = J P^{-1} V_j                      (k_spmm, ilu kernels)
//   H = [V]^T W, W -= [V] H   twice       (k_gram + k_gram_reduce, k_update)
//   W = V_{j+1} R  by CholQR2             (k_gram, k_chol, k_rowmul)
//   Householder update of the block Hessenberg least-squares problem and the
//   per-column residual estimates         (k_hess_step, one CTA, float64)
// The outer loop is the fixed point of Eq. matrix-fixed-point-equation as
// defect correction: R = R(Y) (k_coupled, float64), V = J^{-1} R, Y -= V.
#include "internal.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>

namespace pint {

constexpr int kGramTile = 16;      // rows staged in shared memory per pass
constexpr int kSmallLd = 17;       // reflector pitch (s + 1 <= 17)

// ------------------------------------------------------------- Gram (a5)
// partial[blk][p][k] = sum over this CTA's rows r of V_b[r][i] * W[r][k],
// p = b*s + i. Threads: PT p-lanes x TR row groups; NPT p-values per thread.
template <typename VT, int S, bool EXACT, int NPT>
__global__ void __launch_bounds__(256)
k_gram(int64_t n, int s, int nb, const VT* __restrict__ V, int64_t bstride,
       const VT* __restrict__ W, int64_t rows_per_cta, double* __restrict__ partial) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  VT* T = reinterpret_cast<VT*>(smem_raw);
  const int P = nb * s;
  const int pitch = P + s;
  int PT = 32;
  while (PT < P && PT < 256) PT <<= 1;
  const int TR = 256 / PT;
  const int pg = threadIdx.x % PT, rg = threadIdx.x / PT;
  VT acc[NPT][S];
#pragma unroll
  for (int j = 0; j < NPT; ++j)
#pragma unroll
    for (int k = 0; k < S; ++k) acc[j][k] = VT(0);

  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = (r0 + rows_per_cta < n) ? r0 + rows_per_cta : n;
  for (int64_t tile = r0; tile < r1; tile += kGramTile) {
    const int nrows = (int)((r1 - tile) < kGramTile ? (r1 - tile) : kGramTile);
    const int seg = nrows * s;
    for (int b = 0; b <= nb; ++b) {
      const VT* src = (b < nb ? V + (int64_t)b * bstride : W) + tile * s;
      for (int e = threadIdx.x; e < seg; e += 256) {
        const int rr = e / s, i = e - rr * s;
        T[rr * pitch + b * s + i] = src[e];
      }
    }
    __syncthreads();
    for (int rr = rg; rr < nrows; rr += TR) {
      VT w[S];
#pragma unroll
      for (int k = 0; k < S; ++k) w[k] = (EXACT || k < s) ? T[rr * pitch + P + k] : VT(0);
#pragma unroll
      for (int j = 0; j < NPT; ++j) {
        const int p = pg + j * PT;
        if (p < P) {
          const VT v = T[rr * pitch + p];
#pragma unroll
          for (int k = 0; k < S; ++k) acc[j][k] = fma(v, w[k], acc[j][k]);
        }
      }
    }
    __syncthreads();
  }
  // cross row-group reduction in float64
  double* red = reinterpret_cast<double*>(smem_raw);
  const int E = P * s;
  double* out = partial + (int64_t)blockIdx.x * E;
  if (TR == 1) {
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      const int p = pg + j * PT;
      if (p < P)
#pragma unroll
        for (int k = 0; k < S; ++k)
          if (EXACT || k < s) out[p * s + k] = (double)acc[j][k];
    }
    return;
  }
  // NPT == 1 whenever TR > 1 (P <= 128)
  for (int rgi = 0; rgi < TR; ++rgi) {
    if (rg == rgi && pg < P) {
#pragma unroll
      for (int k = 0; k < S; ++k)
        if (EXACT || k < s)
          red[pg * s + k] = (rgi == 0 ? 0.0 : red[pg * s + k]) + (double)acc[0][k];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < E; e += 256) out[e] = red[e];
}

// ---------------------------------------------------- Gram, TMA pipeline
// Same product over a zero-padded row range [0, n_pad): each CTA streams
// tiles of TR rows of the nb+1 blocks (V_0..V_{nb-1}, W) into shared memory
// with 1-D bulk copies (cp.async.bulk, completion on an mbarrier) through a
// ring of stages (k_gram_bulk below). Waits on the mbarriers are bounded
// (globaltimer); a timeout raises *err and the CTA drains without waiting
// further.
constexpr unsigned long long kMbarBudgetNs = 2000000000ull;

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
      "l"(src), "r"(bytes), "r"(b)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(a), "r"(parity) : "memory");
  return done != 0;
}

// Bounded wait for phase `parity` of an mbarrier. Returns true when the phase
// completed; false when *aborted was raised by another thread of the CTA or
// when `deadline` (globaltimer) passed, in which case it raises *aborted and
// stores `code` into the error word *err. Never traps.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  unsigned long long deadline,
                                                  volatile int* aborted, int* err, int code) {
  while (!mbar_try_wait(bar, parity)) {
    if (*aborted) return false;
    if (gtimer() > deadline) {
      *aborted = 1;
      atomicExch(err, code);
      return false;
    }
  }
  return true;
}

// Thread work unit: Q consecutive basis columns (b, i0..i0+Q-1) x all S
// columns of W, kept in Q*S register accumulators; per row one Q-wide and
// S/4 four-wide shared loads feed Q*S FMAs. Each block's stage region is
// padded by kGramPad bytes to spread consecutive quads over the banks.
constexpr int kGramPad = 32;

template <typename VT, int N>
struct VecOf;
template <> struct VecOf<float, 4> { using T = float4; };
template <> struct VecOf<float, 2> { using T = float2; };
template <> struct VecOf<double, 2> { using T = double2; };

template <typename VT, int Q>
__device__ __forceinline__ void lds_q(const VT* p, VT (&v)[Q]) {
  if constexpr (Q % 4 == 0 && sizeof(VT) == 4) {
#pragma unroll
    for (int i = 0; i < Q / 4; ++i) {
      const float4 t = reinterpret_cast<const float4*>(p)[i];
      v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
    }
  } else if constexpr (Q % 2 == 0 && sizeof(VT) == 8) {
#pragma unroll
    for (int i = 0; i < Q / 2; ++i) {
      const double2 t = reinterpret_cast<const double2*>(p)[i];
      v[2 * i] = t.x; v[2 * i + 1] = t.y;
    }
  } else if constexpr (Q == 2 && sizeof(VT) == 4) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = p[i];
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

constexpr int kGramMaxStages = 8;

// Warp-specialised form: NT consumer threads and one producer warp (threads
// NT .. NT+31). The producer fills a ring of ST stages of TR rows of the nb+1
// blocks with 1-D bulk copies (completion on the stage's "full" mbarrier);
// each consumer warp arrives on the stage's "empty" mbarrier when it has
// read the stage, and the producer waits for that before refilling it, so no
// CTA-wide barrier separates the tiles. Every wait is bounded (globaltimer);
// a timeout raises *err, stops the producer and the remaining waits, and the
// producer drains its copies in flight before the CTA reuses the ring.
//
// FUSE: the first update of the second Gram-Schmidt pass is folded in. The
// kernel receives H1 = [V]^T W of the first pass ((nb*s) x s, float64) and,
// for every tile, first forms W1 = W - [V] H1 on the tile's rows from the
// staged blocks (written back to the stage and to Wout, which is W itself:
// each tile of W is copied in once, before it is overwritten), then takes
// the products [V]^T W1 of the tile. One pass over the basis instead of two.
template <typename VT, int S, bool EXACT, int Q, int NQPT, int NT, bool FUSE = false>
__global__ void __launch_bounds__(NT + 32)
k_gram_bulk(int64_t n_pad, int s, int nb, const VT* __restrict__ V, int64_t bstride,
            const VT* __restrict__ W, int64_t rows_per_cta, int TR, int TRG, int ST,
            double* __restrict__ partial, int* __restrict__ err, const double* H1 = nullptr,
            VT* Wout = nullptr) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kGramMaxStages], empty[kGramMaxStages];
  __shared__ int aborted;
  const int P = nb * s;
  const int NQ = P / Q;                                   // quads (Q | s)
  const unsigned blk_bytes = (unsigned)(TR * s * sizeof(VT));
  const unsigned blk_pitch = blk_bytes + kGramPad;
  const unsigned stage_bytes = blk_pitch * (nb + 1);
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = (r0 + rows_per_cta < n_pad) ? r0 + rows_per_cta : n_pad;
  const int ntiles = r1 > r0 ? (int)((r1 - r0) / TR) : 0;
  const int tid = threadIdx.x;
  // FUSE: H1 in the vector precision, pitch S, after the ring
  VT* H1s = reinterpret_cast<VT*>(smem_raw + (((size_t)ST * stage_bytes + 15) & ~(size_t)15));
  if constexpr (FUSE) {
    for (int e = tid; e < P * S; e += blockDim.x) {
      const int p = e / S, k = e - p * S;
      H1s[e] = (k < s) ? (VT)H1[p * s + k] : VT(0);
    }
  }
  if (tid == 0) {
    for (int i = 0; i < ST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], NT / 32);
    }
    aborted = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const unsigned long long deadline = gtimer() + kMbarBudgetNs;
  // consumer mapping: quads q = qbase + j*qstride (j < NQPT), rows rg + m*TRG
  const int qstride = (NQ + NQPT - 1) / NQPT;
  const int qbase = tid % qstride, rg = tid / qstride;
  const bool active = tid < NT && rg < TRG;
  VT acc[NQPT][Q][S];
#pragma unroll
  for (int j = 0; j < NQPT; ++j)
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
      for (int k = 0; k < S; ++k) acc[j][i][k] = VT(0);
  int qoff[NQPT];
#pragma unroll
  for (int j = 0; j < NQPT; ++j) {
    const int q = qbase + j * qstride;
    const int p = q * Q;
    qoff[j] = (q < NQ) ? (int)((p / s) * (blk_pitch / sizeof(VT)) + (p % s)) : -1;
  }
  if (tid >= NT) {
    // ------------------------------------------------------ producer warp
    const int lane = tid - NT;
    int last_t[kGramMaxStages];
    for (int i = 0; i < kGramMaxStages; ++i) last_t[i] = -1;
    for (int t = 0; t < ntiles; ++t) {
      const int st = t % ST;
      if (t >= ST) {            // the consumers have read the stage's previous tile
        bool ok = true;
        if (lane == 0)
          ok = mbar_wait_bounded(&empty[st], (unsigned)((t / ST - 1) & 1), deadline, &aborted,
                                 err, 3);
        if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
      }
      if (*(volatile int*)&aborted) break;
      unsigned char* dst = smem_raw + (size_t)st * stage_bytes;
      if (lane == 0) mbar_expect_tx(&full[st], blk_bytes * (nb + 1));
      __syncwarp();
      const int64_t row = r0 + (int64_t)t * TR;
      for (int b = lane; b <= nb; b += 32) {
        const VT* src = (b < nb ? V + (int64_t)b * bstride : W) + row * s;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bulk_g2s(dst + (size_t)b * blk_pitch, src, blk_bytes, &full[st]);
      }
      last_t[st] = t;
    }
    // every copy issued has landed before the ring's memory is reused below
    // (bounded; after a timeout some stages were never consumed)
    if (lane == 0) {
      const unsigned long long drain = gtimer() + kMbarBudgetNs;
      for (int i = 0; i < ST; ++i)
        if (last_t[i] >= 0)
          while (!mbar_try_wait(&full[i], (unsigned)((last_t[i] / ST) & 1)) && gtimer() < drain) {
          }
    }
  } else {
    // ----------------------------------------------------- consumer warps
    for (int t = 0; t < ntiles; ++t) {
      const int st = t % ST;
      if (!*(volatile int*)&aborted)
        mbar_wait_bounded(&full[st], (unsigned)((t / ST) & 1), deadline, &aborted, err, 3);
      if constexpr (FUSE) {
        // W1 = W - [V] H1 on this tile's rows, a row per consumer thread; the
        // products below read the updated rows after the consumers' barrier,
        // which every consumer thread reaches once per tile whatever happened
        if (!*(volatile int*)&aborted) {
          VT* Tm = reinterpret_cast<VT*>(smem_raw + (size_t)st * stage_bytes);
          VT* Wm = reinterpret_cast<VT*>(smem_raw + (size_t)st * stage_bytes +
                                         (size_t)nb * blk_pitch);
          const int64_t row0 = r0 + (int64_t)t * TR;
          for (int rr = tid; rr < TR; rr += NT) {
            VT acc[S];
#pragma unroll
            for (int k = 0; k < S; ++k) acc[k] = VT(0);
            for (int b = 0; b < nb; ++b) {
              VT v[S];
              const VT* vr = Tm + (size_t)b * (blk_pitch / sizeof(VT)) + rr * s;
              if constexpr (EXACT) {
                lds_q<VT, S>(vr, v);
              } else {
#pragma unroll
                for (int i = 0; i < S; ++i) v[i] = i < s ? vr[i] : VT(0);
              }
              const VT* hb = H1s + b * s * S;
#pragma unroll
              for (int i = 0; i < S; ++i) {
                if (!EXACT && i >= s) break;
#pragma unroll
                for (int k = 0; k < S; ++k) acc[k] = fma(v[i], hb[i * S + k], acc[k]);
              }
            }
#pragma unroll
            for (int k = 0; k < S; ++k) {
              if (!EXACT && k >= s) break;
              const VT w1 = Wm[rr * s + k] - acc[k];
              Wm[rr * s + k] = w1;
              Wout[(row0 + rr) * s + k] = w1;
            }
          }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory");
      }
      if (active && !*(volatile int*)&aborted) {
        const VT* T = reinterpret_cast<const VT*>(smem_raw + (size_t)st * stage_bytes);
        const VT* Wt = reinterpret_cast<const VT*>(smem_raw + (size_t)st * stage_bytes +
                                                   (size_t)nb * blk_pitch);
#pragma unroll 2
        for (int rr = rg; rr < TR; rr += TRG) {
          VT w[S];
          if constexpr (EXACT) {
            lds_q<VT, S>(Wt + rr * S, w);
          } else {
#pragma unroll
            for (int k = 0; k < S; ++k) w[k] = k < s ? Wt[rr * s + k] : VT(0);
          }
#pragma unroll
          for (int j = 0; j < NQPT; ++j) {
            if (qoff[j] >= 0) {
              VT v[Q];
              lds_q<VT, Q>(T + qoff[j] + rr * s, v);
#pragma unroll
              for (int i = 0; i < Q; ++i)
#pragma unroll
                for (int k = 0; k < S; ++k) acc[j][i][k] = fma(v[i], w[k], acc[j][i][k]);
            }
          }
        }
      }
      __syncwarp();
      if ((tid & 31) == 0) mbar_arrive(&empty[st]);
    }
  }
  __syncthreads();
  // the row groups' partial sums, each in its own slot, then summed per entry
  // in row-group order (float64, deterministic)
  double* red = reinterpret_cast<double*>(smem_raw);
  const int E = P * s;
  if (active) {
#pragma unroll
    for (int j = 0; j < NQPT; ++j) {
      if (qoff[j] < 0) continue;
      const int p0 = (qbase + j * qstride) * Q;
#pragma unroll
      for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int k = 0; k < S; ++k)
          if (EXACT || k < s) red[(size_t)rg * E + (p0 + i) * s + k] = (double)acc[j][i][k];
    }
  }
  __syncthreads();
  double* out = partial + (int64_t)blockIdx.x * E;
  for (int e = tid; e < E; e += blockDim.x) {
    double v = 0.0;
    for (int g = 0; g < TRG; ++g) v += red[(size_t)g * E + e];
    out[e] = v;
  }
}

// H[e] = sum_blk partial[blk][e]. One warp per entry: lane l sums blocks
// l, l+32, ... (independent loads in flight), then a fixed shuffle tree; the
// order is fixed, so the result is deterministic.
__global__ void k_gram_reduce_w(int nblk, int E, const double* __restrict__ partial,
                                double* __restrict__ H) {
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= E) return;
  double v = 0.0;
#pragma unroll 4
  for (int b = lane; b < nblk; b += 32) v += partial[(int64_t)b * E + e];
  v = warp_sum(v);
  if (lane == 0) H[e] = v;
}
#define k_gram_reduce_launch(E_, nblk_, partial_, H_, st_) \
  k_gram_reduce_w<<<((E_) + 7) / 8, 256, 0, (st_)>>>((nblk_), (E_), (partial_), (H_))

// one thread per entry (small partial counts: the no-allocation variant)
__global__ void k_gram_reduce(int nblk, int E, const double* __restrict__ partial,
                              double* __restrict__ H) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double v = 0.0;
  for (int b = 0; b < nblk; ++b) v += partial[(int64_t)b * E + e];
  H[e] = v;
}

// Test of the bounded mbarrier wait: one CTA posts an expected transaction
// count of 16 bytes that no copy ever delivers, then waits for the phase
// through mbar_wait_bounded with a deadline `budget_ns` from now. No copy is
// in flight, so the CTA returns as soon as the wait gives up.
__global__ void k_test_mbar_timeout(unsigned long long budget_ns, int* err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int aborted;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    aborted = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar, 16);
  }
  __syncthreads();
  const unsigned long long deadline = gtimer() + budget_ns;
  mbar_wait_bounded(&bar, 0, deadline, &aborted, err, 3);
}

void test_mbar_timeout(double limit_ms, int* err, cudaStream_t st) {
  k_test_mbar_timeout<<<1, 32, 0, st>>>((unsigned long long)(limit_ms * 1e6), err);
  check_launch("k_test_mbar_timeout");
}

static void ensure_partial(pint_ctx ctx, size_t bytes) {
  if (ctx->partial_bytes >= bytes) return;
  if (ctx->d_partial) dfree(ctx, ctx->d_partial, ctx->partial_bytes);
  ctx->d_partial = static_cast<double*>(dalloc(ctx, bytes));
  ctx->partial_bytes = bytes;
}

// H = [V]^T W by k_gram_bulk; with H1 != nullptr the fused form: W <- W -
// [V] H1 first (in place), then H = [V]^T W of the updated W. Returns false,
// launching nothing, when the bulk path does not apply.
template <typename VT>
static bool gram_bulk_t(pint_ctx ctx, int64_t n_pad, int s, int nb, const VT* V, int64_t bstride,
                        const VT* W, double* H, cudaStream_t st, const double* H1 = nullptr,
                        VT* Wout = nullptr) {
  const int P = nb * s;
  const size_t es = sizeof(VT);
  const bool fuse = H1 != nullptr;
  // FUSE stages H1 (P x S in the vector precision) after the ring
  const size_t h1_bytes = fuse ? es * (size_t)P * 16 + 16 : 0;
  if (n_pad % 64 != 0 || (bstride * es) % 16 != 0 ||
      reinterpret_cast<uintptr_t>(V) % 16 != 0 || reinterpret_cast<uintptr_t>(W) % 16 != 0)
    return false;
  // tile rows: the largest power of two <= 1024 dividing n_pad with a stage of
  // at most 48 KB, so a CTA keeps ~200 KB of loads in flight whatever nb and s
  // in copies of at least 1 KB per block
  auto stage_of = [&](int tr) { return (size_t)(nb + 1) * (tr * s * es + kGramPad); };
  int TR = 1024;
  while (TR > 4 && (stage_of(TR) > 66 * 1024 || n_pad % TR != 0)) TR >>= 1;
  if (stage_of(TR) > 66 * 1024 || n_pad % TR != 0) return false;
  const size_t stage_bytes = stage_of(TR);
  if (2 * stage_bytes + h1_bytes > 210 * 1024) return false;
  const int STG = (int)std::max<size_t>(
      2, std::min<size_t>(kGramMaxStages, (210 * 1024 - h1_bytes) / stage_bytes));
  const int E = P * s;
  bool ok = true;
  with_s(s, [&](auto S_, auto E_) {
    constexpr int S = decltype(S_)::value;
    constexpr bool EX = decltype(E_)::value;
    constexpr int Q = EX ? (S >= 4 ? 4 : S) : 1;
    // consumer threads: 512 for float32 blocks of width exactly 8 (measured at 128^3:
    // 3.75 -> 4.10 TB/s, 16 instead of 8 warps hiding the products' FMA and
    // shared-memory latency); 256 elsewhere, where 512 would spill registers
    constexpr int NT = (sizeof(VT) == 4 && S == 8 && EX) ? 512 : 256;
    const int NQ = P / Q;
    const int npt = NQ <= NT ? 1 : NQ <= 2 * NT ? 2 : 4;
    const int qs = (NQ + npt - 1) / npt;
    int TRG = std::max(1, std::min(64, NT / qs));
    while (TRG > 1 && (size_t)TRG * E * 8 > 210 * 1024) TRG >>= 1;
    const size_t smem = std::max((size_t)STG * stage_bytes + h1_bytes, (size_t)TRG * E * 8);
    if (smem > 210 * 1024 || NQ > 1024) {
      ok = false;
      return;
    }
    auto launch = [&](auto kern) {
      smem_attr(kern, smem);
      int per_sm = 0;
      PINT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT + 32, smem));
      int64_t want = std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(1, per_sm) * ctx->num_sms,
                                                            n_pad / TR));
      int64_t rpc = (n_pad + want - 1) / want;
      rpc = ((rpc + TR - 1) / TR) * TR;
      const int nblk = (int)((n_pad + rpc - 1) / rpc);
      ensure_partial(ctx, sizeof(double) * (size_t)nblk * E);
      kern<<<nblk, NT + 32, smem, st>>>(n_pad, s, nb, V, bstride, W, rpc, TR, TRG, STG,
                                        ctx->d_partial, ctx->d_flag, H1, Wout);
      check_launch("k_gram_bulk");
      k_gram_reduce_launch(E, nblk, ctx->d_partial, H, st);
      check_launch("k_gram_reduce");
    };
    // with Q = 4 there are at most 256 quads (P <= 1024): one per thread
    if (fuse) {
      // float64 at s = 16 keeps the separate launches: the update's row and
      // the products' accumulators do not fit in registers together
      if constexpr (sizeof(VT) == 8 && S == 16) {
        ok = false;
        return;
      } else {
        if constexpr (Q == 4) launch(k_gram_bulk<VT, S, EX, Q, 1, NT, true>);
        else if (npt == 1) launch(k_gram_bulk<VT, S, EX, Q, 1, NT, true>);
        else if (npt == 2) launch(k_gram_bulk<VT, S, EX, Q, 2, NT, true>);
        else launch(k_gram_bulk<VT, S, EX, Q, 4, NT, true>);
      }
    } else {
      if constexpr (Q == 4) launch(k_gram_bulk<VT, S, EX, Q, 1, NT>);
      else if (npt == 1) launch(k_gram_bulk<VT, S, EX, Q, 1, NT>);
      else if (npt == 2) launch(k_gram_bulk<VT, S, EX, Q, 2, NT>);
      else launch(k_gram_bulk<VT, S, EX, Q, 4, NT>);
    }
  });
  if (!ok) return false;
  ctx->launches += 2;
  return true;
}

template <typename VT>
static void gram_t(pint_ctx ctx, int64_t n, int s, int nb, const VT* V, int64_t bstride,
                   const VT* W, double* H, cudaStream_t st, int fam = PF_GRAM,
                   int64_t n_pad = 0) {
  const int P = nb * s;
  ProfScope ps(ctx, fam, sizeof(VT) * (double)(nb + 1) * n * s, 2.0 * n * nb * s * s, st);
  if (n_pad > 0 && gram_bulk_t<VT>(ctx, n_pad, s, nb, V, bstride, W, H, st)) return;
  PINT_REQUIRE(P <= 1024, PINT_ERR_INVALID, "Gram block too wide (nb*s > 1024)");
  int PT = 32;
  while (PT < P && PT < 256) PT <<= 1;
  const int npt = (P + PT - 1) / PT;
  const int64_t want = std::max<int64_t>(1, std::min<int64_t>(4LL * ctx->num_sms, (n + 63) / 64));
  int64_t rpc = (n + want - 1) / want;
  rpc = std::max<int64_t>(kGramTile, ((rpc + kGramTile - 1) / kGramTile) * kGramTile);
  const int nblk = (int)((n + rpc - 1) / rpc);
  const int E = P * s;
  ensure_partial(ctx, sizeof(double) * (size_t)nblk * E);
  const size_t tile_bytes = sizeof(VT) * kGramTile * (P + s);
  const size_t red_bytes = sizeof(double) * E;
  const size_t smem = std::max(tile_bytes, (PT < 256 ? red_bytes : (size_t)0));
  with_s(s, [&](auto S_, auto E_) {
    constexpr int S = decltype(S_)::value;
    constexpr bool EX = decltype(E_)::value;
    auto launch = [&](auto kern) {
      smem_attr(kern, smem);
      kern<<<nblk, 256, smem, st>>>(n, s, nb, V, bstride, W, rpc, ctx->d_partial);
    };
    if (npt == 1) launch(k_gram<VT, S, EX, 1>);
    else if (npt == 2) launch(k_gram<VT, S, EX, 2>);
    else launch(k_gram<VT, S, EX, 4>);
  });
  check_launch("k_gram");
  k_gram_reduce_launch(E, nblk, ctx->d_partial, H, st);
  check_launch("k_gram_reduce");
  ctx->launches += 2;
}

void launch_gram(pint_ctx ctx, int precision, int64_t n, int s, int nb, const void* V,
                 int64_t bstride, const void* W, double* H, cudaStream_t st, int64_t n_pad) {
  if (precision == PINT_FP64)
    gram_t<double>(ctx, n, s, nb, (const double*)V, bstride, (const double*)W, H, st, PF_GRAM,
                   n_pad);
  else
    gram_t<float>(ctx, n, s, nb, (const float*)V, bstride, (const float*)W, H, st, PF_GRAM,
                  n_pad);
}

// ------------------------------------------------------- block update (a6)
// MODE 0: W -= V H ; 1: W = V H ; 2: W += V H. H ((nb*s) x s, float64) is
// staged in shared memory in the vector precision with pitch S.
template <typename VT, int S, bool EXACT, int MODE>
__global__ void __launch_bounds__(256)
k_update(int64_t n, int s, int nb, const VT* __restrict__ V, int64_t bstride,
         const double* __restrict__ H, VT* __restrict__ W) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  VT* Hs = reinterpret_cast<VT*>(smem_raw);
  const int P = nb * s;
  for (int e = threadIdx.x; e < P * S; e += blockDim.x) {
    const int p = e / S, k = e - p * S;
    Hs[e] = (k < s) ? (VT)H[p * s + k] : VT(0);
  }
  __syncthreads();
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    VT acc[S];
#pragma unroll
    for (int k = 0; k < S; ++k) acc[k] = VT(0);
    // unrolled so that the loads of later blocks issue ahead of this block's
    // FMAs (5.44 -> 5.57 TB/s at 128^3, s = 8, float32)
#pragma unroll 4
    for (int b = 0; b < nb; ++b) {
      VT v[S];
      load_row<S, EXACT>(V + (int64_t)b * bstride + r * s, s, v);
      const VT* hb = Hs + b * s * S;
#pragma unroll
      for (int i = 0; i < S; ++i) {
        if (!EXACT && i >= s) break;
#pragma unroll
        for (int k = 0; k < S; ++k) acc[k] = fma(v[i], hb[i * S + k], acc[k]);
      }
    }
    VT* wr = W + r * s;
    if constexpr (MODE == 1) {
      store_row<S, EXACT>(wr, s, acc);
    } else {
      VT w[S];
      load_row<S, EXACT>(wr, s, w);
#pragma unroll
      for (int k = 0; k < S; ++k) w[k] = (MODE == 0) ? w[k] - acc[k] : w[k] + acc[k];
      store_row<S, EXACT>(wr, s, w);
    }
  }
}

template <typename VT>
static void update_t(pint_ctx ctx, int64_t n, int s, int nb, const VT* V, int64_t bstride,
                     const double* H, VT* W, int mode, cudaStream_t st) {
  const int P = nb * s;
  ProfScope ps(ctx, PF_UPDATE, sizeof(VT) * (double)n * s * (nb + (mode == 1 ? 1 : 2)),
               2.0 * n * nb * s * s, st);
  with_s(s, [&](auto S_, auto E_) {
    constexpr int S = decltype(S_)::value;
    constexpr bool EX = decltype(E_)::value;
    const size_t smem = sizeof(VT) * (size_t)P * S;
    const unsigned g = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(4LL * ctx->num_sms, (n + 255) / 256));
    auto launch = [&](auto kern) {
      smem_attr(kern, smem);
      kern<<<g, 256, smem, st>>>(n, s, nb, V, bstride, H, W);
    };
    if (mode == 0) launch(k_update<VT, S, EX, 0>);
    else if (mode == 1) launch(k_update<VT, S, EX, 1>);
    else launch(k_update<VT, S, EX, 2>);
  });
  check_launch("k_update");
  ctx->launches += 1;
}

void launch_update(pint_ctx ctx, int precision, int64_t n, int s, int nb, const void* V,
                   int64_t bstride, const double* H, void* W, int mode, cudaStream_t st) {
  if (precision == PINT_FP64)
    update_t<double>(ctx, n, s, nb, (const double*)V, bstride, H, (double*)W, mode, st);
  else
    update_t<float>(ctx, n, s, nb, (const float*)V, bstride, H, (float*)W, mode, st);
}

// W <- W - [V] H1, then H2 = [V]^T W: the first update and the second Gram
// product of block CGS2, in one pass over the basis (k_gram_bulk<...,
// FUSE>) for float32 blocks of width s <= 4 on the bulk Gram path, else as
// the two separate launches. Measured at 128^3 (whole slab solves, float32
// inner): the fused pass gains 4, 3 and 2.6 % at s = 1, 2, 4 and loses
// 0.4 % at s = 8, 5 % at s = 16 and 12 % in float64 at s = 8: its update
// phase runs one row per thread on the eight consumer warps, serialised with
// the products by a barrier, which the saved read of the basis pays for only
// while s is small.
template <typename VT>
static void update_gram_t(pint_ctx ctx, int64_t n, int s, int nb, const VT* V, int64_t bstride,
                          const double* H1, VT* W, double* H2, cudaStream_t st, int64_t n_pad) {
  if (n_pad > 0 && ctx->gram_fuse && sizeof(VT) == 4 && s <= 4) {
    ProfScope ps(ctx, PF_GRAM, sizeof(VT) * (double)(nb + 2) * n * s, 4.0 * n * nb * s * s, st);
    if (gram_bulk_t<VT>(ctx, n_pad, s, nb, V, bstride, W, H2, st, H1, W)) return;
    ps.cancel();
  }
  update_t<VT>(ctx, n, s, nb, V, bstride, H1, W, 0, st);
  gram_t<VT>(ctx, n, s, nb, V, bstride, W, H2, st, PF_GRAM, n_pad);
}

void launch_update_gram(pint_ctx ctx, int precision, int64_t n, int s, int nb, const void* V,
                        int64_t bstride, const double* H1, void* W, double* H2, cudaStream_t st,
                        int64_t n_pad) {
  if (precision == PINT_FP64)
    update_gram_t<double>(ctx, n, s, nb, (const double*)V, bstride, H1, (double*)W, H2, st,
                          n_pad);
  else
    update_gram_t<float>(ctx, n, s, nb, (const float*)V, bstride, H1, (float*)W, H2, st, n_pad);
}

// ------------------------------------------------------------ CholQR (a7)
// Upper Cholesky G = R^T R in natural order with deflation (pivot <=
// defl * G_kk or G_kk <= 0 -> zero row of R); Rinv with Q = W Rinv, zero
// columns for deflated k. One CTA of 256 threads, s <= 16.
__global__ void k_chol(int s, const double* __restrict__ G, double defl, double* __restrict__ R,
                       double* __restrict__ Rinv, int* __restrict__ defl_count) {
  __shared__ double Gs[kMaxS][kMaxS + 1];
  __shared__ double Rs[kMaxS][kMaxS + 1];
  __shared__ double g0[kMaxS];
  __shared__ double dinv[kMaxS];     // 1 / R[k][k] (0 when deflated)
  __shared__ int dead[kMaxS];
  const int t = threadIdx.x, i = t / kMaxS, j = t % kMaxS;
  if (i < s && j < s) {
    Gs[i][j] = G[i * s + j];
    Rs[i][j] = 0.0;
  }
  if (t < s) g0[t] = G[t * s + t];
  __syncthreads();
  for (int k = 0; k < s; ++k) {
    __shared__ double piv;
    if (t == 0) {
      const double d = Gs[k][k];
      const bool isdead = !(g0[k] > 0.0) || !(d > defl * g0[k]);
      dead[k] = isdead ? 1 : 0;
      piv = isdead ? 0.0 : sqrt(d);
      dinv[k] = isdead ? 0.0 : 1.0 / piv;     // the one division of step k
      if (isdead && defl_count) atomicAdd(defl_count, 1);
    }
    __syncthreads();
    if (t < s && t >= k) Rs[k][t] = dead[k] ? 0.0 : (t == k ? piv : Gs[k][t] * dinv[k]);
    __syncthreads();
    if (i < s && j < s && i > k && j > k) Gs[i][j] -= Rs[k][i] * Rs[k][j];
    __syncthreads();
  }
  if (i < s && j < s) R[i * s + j] = Rs[i][j];
  // row t of Rinv: Rinv[t][k] = ((t==k) - sum_{c<k} Rinv[t][c] R[c][k]) / R[k][k]
  if (t < s) {
    double row[kMaxS];
    for (int k = 0; k < s; ++k) {
      double v = 0.0;
      if (!dead[k]) {
        v = (t == k) ? 1.0 : 0.0;
        for (int c = 0; c < k; ++c) v -= row[c] * Rs[c][k];
        v *= dinv[k];
      }
      row[k] = v;
    }
    for (int k = 0; k < s; ++k) Rinv[t * s + k] = row[k];
  }
}

// W[r] <- W[r] * Ri (s x s), in place: each thread owns a row.
template <typename VT, int S, bool EXACT>
__global__ void __launch_bounds__(256)
k_rowmul(int64_t n, int s, VT* __restrict__ W, const double* __restrict__ Ri) {
  __shared__ VT Rs[S * S];
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
    const int i = e / S, k = e % S;
    Rs[e] = (i < s && k < s) ? (VT)Ri[i * s + k] : VT(0);
  }
  __syncthreads();
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    VT w[S], o[S];
    load_row<S, EXACT>(W + r * s, s, w);
#pragma unroll
    for (int k = 0; k < S; ++k) o[k] = VT(0);
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int k = i; k < S; ++k) o[k] = fma(w[i], Rs[i * S + k], o[k]);
    store_row<S, EXACT>(W + r * s, s, o);
  }
}

// C = A B for s x s row-major matrices (one CTA).
__global__ void k_small_mm(int s, const double* __restrict__ A, const double* __restrict__ B,
                           double* __restrict__ C) {
  const int t = threadIdx.x, i = t / kMaxS, j = t % kMaxS;
  if (i >= s || j >= s) return;
  double v = 0.0;
  for (int k = 0; k < s; ++k) v += A[i * s + k] * B[k * s + j];
  C[i * s + j] = v;
}

struct CholScratch {
  double* G;
  double* R1;
  double* R2;
  double* Rinv;
};

static CholScratch chol_scratch(pint_ctx ctx) {
  double* b = ctx->d_small + kSmallChol;
  return {b, b + 256, b + 512, b + 768};
}

template <typename VT>
static void cholqr_pass(pint_ctx ctx, int64_t n, int s, VT* W, double* R, double defl,
                        int* defl_count, cudaStream_t st, int64_t n_pad) {
  CholScratch cs = chol_scratch(ctx);
  gram_t<VT>(ctx, n, s, 1, W, 0, W, cs.G, st, PF_CHOLQR, n_pad);
  ProfScope ps(ctx, PF_CHOLQR, 2.0 * sizeof(VT) * n * s, 1.0 * n * s * s, st);
  k_chol<<<1, 256, 0, st>>>(s, cs.G, defl, R, cs.Rinv, defl_count);
  check_launch("k_chol");
  with_s(s, [&](auto S_, auto E_) {
    constexpr int S = decltype(S_)::value;
    constexpr bool EX = decltype(E_)::value;
    const unsigned g = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(8LL * ctx->num_sms, (n + 255) / 256));
    k_rowmul<VT, S, EX><<<g, 256, 0, st>>>(n, s, W, cs.Rinv);
  });
  check_launch("k_rowmul");
  ctx->launches += 2;
}

// Streaming self-Gram for narrow blocks (S <= 8): G = W^T W (upper triangle
// accumulated per thread over its rows, float64 across threads and CTAs).
// SCALE: first W[r] <- W[r] Rinv (written back), then accumulate the new row:
// the scaling of one CholQR pass fused with the Gram of the next.
template <typename VT, int S, bool SCALE>
__global__ void __launch_bounds__(256)
k_syrk(int64_t n, VT* __restrict__ W, const double* __restrict__ Ri,
       double* __restrict__ partial) {
  constexpr int NT = S * (S + 1) / 2;
  __shared__ VT Rs[S * S];
  __shared__ double red[8][NT];
  if (SCALE) {
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) Rs[e] = (VT)Ri[e];
    __syncthreads();
  }
  VT acc[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) acc[t] = VT(0);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    VT w[S];
    load_row<S, true>(W + r * S, S, w);
    if (SCALE) {
      VT o[S];
#pragma unroll
      for (int k = 0; k < S; ++k) o[k] = VT(0);
#pragma unroll
      for (int i = 0; i < S; ++i)
#pragma unroll
        for (int k = i; k < S; ++k) o[k] = fma(w[i], Rs[i * S + k], o[k]);
      store_row<S, true>(W + r * S, S, o);
#pragma unroll
      for (int k = 0; k < S; ++k) w[k] = o[k];
    }
    int t = 0;
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int k = i; k < S; ++k) {
        acc[t] = fma(w[i], w[k], acc[t]);
        ++t;
      }
  }
  // warp reduction in the vector precision (float64 arithmetic is scarce),
  // float64 across warps and CTAs
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const VT v = warp_sum(acc[t]);
    if (lane == 0) red[warp][t] = (double)v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NT; t += blockDim.x) {
    double v = 0.0;
    for (int w8 = 0; w8 < 8; ++w8) v += red[w8][t];
    // expand the upper triangle to the full S x S partial
    int i = 0, rem = t;
    while (rem >= S - i) {
      rem -= S - i;
      ++i;
    }
    const int k = i + rem;
    partial[(int64_t)blockIdx.x * S * S + i * S + k] = v;
    partial[(int64_t)blockIdx.x * S * S + k * S + i] = v;
  }
}

template <typename VT, int S>
static void syrk_t(pint_ctx ctx, int64_t n, VT* W, const double* Rinv, double* G, bool scale,
                   cudaStream_t st) {
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(4LL * ctx->num_sms, (n + 255) / 256));
  ensure_partial(ctx, sizeof(double) * (size_t)nblk * S * S);
  ProfScope ps(ctx, PF_CHOLQR, sizeof(VT) * (double)n * S * (scale ? 2 : 1),
               (double)n * S * S * (scale ? 2 : 1), st);
  if (scale)
    k_syrk<VT, S, true><<<nblk, 256, 0, st>>>(n, W, Rinv, ctx->d_partial);
  else
    k_syrk<VT, S, false><<<nblk, 256, 0, st>>>(n, W, Rinv, ctx->d_partial);
  check_launch("k_syrk");
  k_gram_reduce_launch(S * S, nblk, ctx->d_partial, G, st);
  check_launch("k_gram_reduce");
  ctx->launches += 2;
}

// CholQR2 for S in {1, 2, 4, 8}: syrk -> chol -> syrk(scale) -> chol -> scale.
template <typename VT, int S>
static void cholqr2_narrow(pint_ctx ctx, int64_t n, VT* W, double* R, double defl,
                           int* defl_count, cudaStream_t st) {
  CholScratch cs = chol_scratch(ctx);
  syrk_t<VT, S>(ctx, n, W, nullptr, cs.G, false, st);
  {
    ProfScope ps(ctx, PF_CHOLQR, 0.0, 1.0 * S * S * S, st);
    k_chol<<<1, 256, 0, st>>>(S, cs.G, defl, cs.R1, cs.Rinv, defl_count);
    check_launch("k_chol");
  }
  syrk_t<VT, S>(ctx, n, W, cs.Rinv, cs.G, true, st);
  ProfScope ps(ctx, PF_CHOLQR, 2.0 * sizeof(VT) * n * S, 1.0 * n * S * S, st);
  k_chol<<<1, 256, 0, st>>>(S, cs.G, defl, cs.R2, cs.Rinv, defl_count);
  check_launch("k_chol");
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(8LL * ctx->num_sms, (n + 255) / 256));
  k_rowmul<VT, S, true><<<g, 256, 0, st>>>(n, S, W, cs.Rinv);
  check_launch("k_rowmul");
  k_small_mm<<<1, 256, 0, st>>>(S, cs.R2, cs.R1, R);
  check_launch("k_small_mm");
  ctx->launches += 4;
}

void cholqr2(pint_ctx ctx, int precision, int64_t n, int s, void* W, double* R,
             int* defl_count, cudaStream_t st, int64_t n_pad) {
  CholScratch cs = chol_scratch(ctx);
  const double defl = precision == PINT_FP64 ? 1e-14 : 1e-8;
  if (s == 1 || s == 2 || s == 4 || s == 8) {
    auto run = [&](auto tag) {
      using VT = decltype(tag);
      VT* w = static_cast<VT*>(W);
      switch (s) {
        case 1: cholqr2_narrow<VT, 1>(ctx, n, w, R, defl, defl_count, st); break;
        case 2: cholqr2_narrow<VT, 2>(ctx, n, w, R, defl, defl_count, st); break;
        case 4: cholqr2_narrow<VT, 4>(ctx, n, w, R, defl, defl_count, st); break;
        default: cholqr2_narrow<VT, 8>(ctx, n, w, R, defl, defl_count, st); break;
      }
    };
    if (precision == PINT_FP64) run(double(0));
    else run(float(0));
    return;
  }
  if (precision == PINT_FP64) {
    cholqr_pass<double>(ctx, n, s, (double*)W, cs.R1, defl, defl_count, st, n_pad);
    cholqr_pass<double>(ctx, n, s, (double*)W, cs.R2, defl, defl_count, st, n_pad);
  } else {
    cholqr_pass<float>(ctx, n, s, (float*)W, cs.R1, defl, defl_count, st, n_pad);
    cholqr_pass<float>(ctx, n, s, (float*)W, cs.R2, defl, defl_count, st, n_pad);
  }
  ProfScope ps(ctx, PF_CHOLQR, 0.0, 2.0 * s * s * s, st);
  k_small_mm<<<1, 256, 0, st>>>(s, cs.R2, cs.R1, R);
  check_launch("k_small_mm");
  ctx->launches += 1;
}

// ---------------------------------------------- block Hessenberg (a8)
// Column block j: [H1 + H2 ; Rn] ((j+2)s x s) -> apply the js earlier
// reflectors (k_hess_old, one CTA per column: the columns are independent
// and the float64 work of one SM is the limit), then make s new reflectors
// of length s+1, rotate Gr, write the per-column residual estimates and
// flag = {all converged, non-finite} (k_hess_step, one CTA).

// sum over the lanes 0..15 (all others hold 0 or are not read)
__device__ __forceinline__ double half_warp_sum(double v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA l: column l of the block, staged with the earlier reflectors in shared
// memory; lane r < s+1 holds row c + r of reflector c's window.
__global__ void __launch_bounds__(32)
k_hess_old(int j, int s, int ldh, const double* __restrict__ H1, const double* __restrict__ H2,
           const double* __restrict__ Rn, double* __restrict__ Hb,
           const double* __restrict__ refl) {
  extern __shared__ double hs[];
  const int l = blockIdx.x, lane = threadIdx.x;
  const int L = (j + 2) * s, top = (j + 1) * s;
  double* cl = hs;                   // the column, L rows
  double* rs = hs + L;               // js reflectors, pitch kSmallLd
  for (int row = lane; row < L; row += 32)
    cl[row] = row < top ? H1[row * s + l] + H2[row * s + l] : Rn[(row - top) * s + l];
  for (int idx = lane; idx < j * s * kSmallLd; idx += 32) rs[idx] = refl[idx];
  __syncwarp();
  const bool act = lane <= s;
  if (s < 16) {
    for (int c = 0; c < j * s; ++c) {
      const double v = act ? rs[c * kSmallLd + lane] : 0.0;
      const double x = act ? cl[c + lane] : 0.0;
      const double d = half_warp_sum(v * x);
      if (act) cl[c + lane] = x - 2.0 * v * d;
      __syncwarp();
    }
  } else {
    for (int c = 0; c < j * s; ++c) {
      const double v = act ? rs[c * kSmallLd + lane] : 0.0;
      const double x = act ? cl[c + lane] : 0.0;
      const double d = warp_sum(v * x);
      if (act) cl[c + lane] = x - 2.0 * v * d;
      __syncwarp();
    }
  }
  for (int row = lane; row < L; row += 32) Hb[(int64_t)(j * s + l) * ldh + row] = cl[row];
}

// One CTA of 512 threads; warp l owns column l (already rotated by the
// earlier reflectors, read from Hb).
__global__ void __launch_bounds__(512)
k_hess_step(int j, int s, int ldh, double* __restrict__ Hb, double* __restrict__ refl,
            double* __restrict__ Gr, const double* __restrict__ target, double* __restrict__ est,
            int* __restrict__ flag) {
  extern __shared__ double col[];
  __shared__ double vcur[32];
  const int L = (j + 2) * s;
  const int top = (j + 1) * s;
  for (int idx = threadIdx.x; idx < s * L; idx += blockDim.x) {
    const int l = idx / L, row = idx - l * L;
    col[idx] = Hb[(int64_t)(j * s + l) * ldh + row];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool act = lane <= s;
  for (int l = 0; l < s; ++l) {
    const int c = j * s + l;
    if (warp == l) {
      double* cl = col + l * L;
      const double x = act ? cl[c + lane] : 0.0;
      const double nrm = sqrt(warp_sum(x * x));
      const double x0 = __shfl_sync(0xffffffffu, x, 0);
      const double beta = x0 >= 0.0 ? -nrm : nrm;
      double v = x - (lane == 0 ? beta : 0.0);
      const double vn = sqrt(warp_sum(v * v));
      v = (vn > 0.0 && act) ? v / vn : 0.0;
      vcur[lane] = v;
      if (act) refl[c * kSmallLd + lane] = v;
      if (act) cl[c + lane] = (lane == 0) ? (nrm > 0.0 ? beta : 0.0) : 0.0;
    }
    __syncthreads();
    if (warp < s) {
      const double v = vcur[lane];
      if (warp > l) {
        double* cl = col + warp * L;
        const double x = act ? cl[c + lane] : 0.0;
        const double d = warp_sum(v * x);
        if (act) cl[c + lane] = x - 2.0 * v * d;
      }
      const double g = act ? Gr[(c + lane) * s + warp] : 0.0;
      const double d = warp_sum(v * g);
      if (act) Gr[(c + lane) * s + warp] = g - 2.0 * v * d;
    }
    __syncthreads();
  }
  if (warp < s) {
    const double g = lane < s ? Gr[(top + lane) * s + warp] : 0.0;
    const double e = sqrt(warp_sum(g * g));
    if (lane == 0) est[warp] = e;
  }
  for (int idx = threadIdx.x; idx < s * L; idx += blockDim.x) {
    const int l = idx / L, row = idx - l * L;
    Hb[(int64_t)(j * s + l) * ldh + row] = col[idx];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int conv = 1, bad = 0;
    for (int k = 0; k < s; ++k) {
      const double e = est[k];
      if (!isfinite(e)) bad = 1;
      if (!(e <= target[k])) conv = 0;
    }
    flag[0] = conv;
    flag[1] = bad;
  }
}

// Gr = [S ; 0] for a new cycle ((m+1)s x s)
__global__ void k_gr_init(int rows, int s, const double* __restrict__ S, double* __restrict__ Gr) {
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < rows * s; e += blockDim.x * gridDim.x)
    Gr[e] = e < s * s ? S[e] : 0.0;
}

// Back substitution Rt Y = Gr[0:kd] with the upper triangle stored in Hb
// (column-major, leading dimension ldh); tiny pivots give zero rows of Y.
__global__ void __launch_bounds__(512)
k_backsolve(int kd, int s, int ldh, const double* __restrict__ Hb, const double* __restrict__ Gr,
            double* __restrict__ Y) {
  extern __shared__ double Gs[];
  __shared__ double ybuf[kMaxS];
  __shared__ double scale;
  for (int e = threadIdx.x; e < kd * s; e += blockDim.x) Gs[e] = Gr[e];
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < kd; ++i) m = fmax(m, fabs(Hb[(int64_t)i * ldh + i]));
    scale = m;
  }
  __syncthreads();
  for (int i = kd - 1; i >= 0; --i) {
    const double rii = Hb[(int64_t)i * ldh + i];
    if (threadIdx.x < s) {
      const double y = fabs(rii) <= 1e-300 + 1e-14 * scale ? 0.0 : Gs[i * s + threadIdx.x] / rii;
      ybuf[threadIdx.x] = y;
      Y[i * s + threadIdx.x] = y;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < i * s; e += blockDim.x) {
      const int r = e / s, k = e - r * s;
      Gs[e] -= Hb[(int64_t)i * ldh + r] * ybuf[k];
    }
    __syncthreads();
  }
}

// X += V (elementwise, n*s)
template <typename VT>
__global__ void k_axpy(int64_t ne, const VT* __restrict__ V, VT* __restrict__ X) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ne) X[i] += V[i];
}

// ------------------------------------------------------- work buffers
struct KrylovWork {
  int64_t n = 0;
  int s = 0, m = 0, prec = -1;
  size_t es = 0;
  void* V = nullptr;     // (m+1) blocks of n*s
  void* Zt = nullptr;    // n*s temp
  void* Xk = nullptr;    // n*s Krylov solution
  void* Rs = nullptr;    // n*s scaled inner right-hand side
  double* R64 = nullptr; // n*s outer residual
  double* Rsub = nullptr; // n*s trailing columns of R64 (narrowed inner solves)
  double* Hg1 = nullptr;
  double* Hg2 = nullptr;
  double* Rn = nullptr;
  double* S = nullptr;
  double* Hb = nullptr;
  double* refl = nullptr;
  double* Gr = nullptr;
  double* Yls = nullptr;
  double* target = nullptr;
  double* est = nullptr;
  double* rnorm = nullptr;
  double* fnorm = nullptr;
  int* flag = nullptr;
  int* defl = nullptr;
  int64_t n_pad = 0;     // rows per basis block (multiple of 64)
  int64_t bs = 0;        // basis block stride in elements (n_pad * s)
  size_t bytes = 0;
  std::vector<std::pair<void*, size_t>> allocs;
};

static void* walloc(pint_ctx ctx, KrylovWork* w, size_t bytes) {
  void* p = dalloc(ctx, bytes);
  w->allocs.push_back({p, bytes});
  return p;
}

void free_work(pint_op op) {
  if (!op->work) return;
  for (auto& a : op->work->allocs) dfree(op->ctx, a.first, a.second);
  delete op->work;
  op->work = nullptr;
}

static KrylovWork* ensure_work(pint_op op, int prec, int m) {
  const int s = op->s;
  KrylovWork* w = op->work;
  if (w && w->n == op->n && w->s >= s && w->m >= m && w->prec == prec) return w;
  free_work(op);
  w = new KrylovWork();
  op->work = w;
  w->n = op->n;
  w->s = s;
  w->m = m;
  w->prec = prec;
  w->es = prec == PINT_FP64 ? 8 : 4;
  pint_ctx ctx = op->ctx;
  const size_t ns = (size_t)op->n * s;
  // basis blocks hold n_pad = 64 * ceil(n / 64) rows; the extra rows stay
  // zero (nothing writes them), which lets the Gram products stream whole
  // 16-byte-aligned tiles with bulk copies
  w->n_pad = ((op->n + 63) / 64) * 64;
  w->bs = w->n_pad * s;
  try {
    w->V = walloc(ctx, w, w->es * (size_t)w->bs * (m + 1));
    PINT_CUDA(cudaMemset(w->V, 0, w->es * (size_t)w->bs * (m + 1)));
    w->Zt = walloc(ctx, w, w->es * ns);
    w->Xk = walloc(ctx, w, w->es * ns);
    w->Rs = walloc(ctx, w, w->es * ns);
    w->R64 = (double*)walloc(ctx, w, 8 * ns);
    w->Rsub = (double*)walloc(ctx, w, 8 * ns);
    const size_t rows = (size_t)(m + 1) * s;
    w->Hg1 = (double*)walloc(ctx, w, 8 * rows * s);
    w->Hg2 = (double*)walloc(ctx, w, 8 * rows * s);
    w->Rn = (double*)walloc(ctx, w, 8 * s * s);
    w->S = (double*)walloc(ctx, w, 8 * s * s);
    w->Hb = (double*)walloc(ctx, w, 8 * rows * (size_t)m * s);
    w->refl = (double*)walloc(ctx, w, 8 * (size_t)m * s * kSmallLd);
    w->Gr = (double*)walloc(ctx, w, 8 * rows * s);
    w->Yls = (double*)walloc(ctx, w, 8 * rows * s);
    w->target = (double*)walloc(ctx, w, 8 * kMaxS);
    w->est = (double*)walloc(ctx, w, 8 * kMaxS);
    w->rnorm = (double*)walloc(ctx, w, 8 * kMaxS);
    w->fnorm = (double*)walloc(ctx, w, 8 * kMaxS);
    w->flag = (int*)walloc(ctx, w, 64);
    w->defl = (int*)walloc(ctx, w, 64);
    // Gram partials for the widest block ((m+1) s) at the largest grid
    ensure_partial(ctx, sizeof(double) * 4 * (size_t)ctx->num_sms * rows * s);
  } catch (...) {
    free_work(op);
    throw;
  }
  return w;
}

// --------------------------------------------------------- inner solve
// Block GMRES(m) on J Xk = Rs (unit columns) in precision VT. With Jacobi the
// matrix is the column-scaled J D^{-1} and Xk is the scaled unknown; with
// ILU(0) the preconditioner is applied to every basis block and to the final
// combination. Returns Arnoldi steps taken.
static InnerResult gmres(pint_op op, const pint_opts* o, KrylovWork* w, cudaStream_t st) {
  pint_ctx ctx = op->ctx;
  const int64_t n = op->n;
  const int s = op->s, m = o->restart, prec = o->precision;
  const int vprec = prec == PINT_FP64 ? PINT_FP64 : PINT_FP32;
  const bool jac = o->precond == PINT_PC_JACOBI;
  const bool ilu = o->precond == PINT_PC_ILU0;
  const int64_t bs = w->bs;        // padded block stride of the basis
  const int64_t ns = n * s;        // elements of an unpadded block vector
  const int64_t np = w->n_pad;
  const size_t es = w->es;
  auto Vb = [&](int b) { return (void*)((char*)w->V + (size_t)b * bs * es); };
  const int ldh = (m + 1) * s;
  // targets: inner_tol (columns are unit or zero)
  {
    double t[kMaxS];
    for (int k = 0; k < s; ++k) t[k] = o->inner_tol;
    PINT_CUDA(cudaMemcpyAsync(w->target, t, 8 * s, cudaMemcpyHostToDevice, st));
  }
  if (s < w->s && np > n)     // narrower than the allocation: rows n..n_pad of a
    for (int b = 0; b <= m; ++b)  // block now overlap old data; the Gram tiles read them
      PINT_CUDA(cudaMemsetAsync((char*)Vb(b) + es * (size_t)ns, 0, es * (size_t)(np - n) * s, st));
  PINT_CUDA(cudaMemsetAsync(w->Xk, 0, es * ns, st));
  PINT_CUDA(cudaMemsetAsync(w->defl, 0, 64, st));
  PINT_CUDA(cudaMemcpyAsync(Vb(0), w->Rs, es * ns, cudaMemcpyDeviceToDevice, st));
  InnerResult res{0, 0, false, 0};
  const size_t hess_smem = 8 * (size_t)s * (m + 1) * s;
  const size_t old_smem = 8 * ((size_t)(m + 1) * s + (size_t)m * s * kSmallLd);
  const size_t back_smem = 8 * (size_t)m * s * s;
  smem_attr(k_hess_step, hess_smem);
  smem_attr(k_hess_old, old_smem);
  smem_attr(k_backsolve, back_smem);
  // One Arnoldi step: W = J P^-1 V_j, BCGS2 against V_0..V_j, CholQR2, the
  // Hessenberg column block and the flags copied to the host.
  auto arnoldi_step = [&](int j, cudaStream_t sx) {
    if (ilu) {
      ilu_apply(op, prec, Vb(j), w->Zt, sx);
      launch_inner_spmm(op, prec, false, w->Zt, Vb(j + 1), nullptr, sx);
    } else {
      launch_inner_spmm(op, prec, jac, Vb(j), Vb(j + 1), nullptr, sx);
    }
    launch_gram(ctx, vprec, n, s, j + 1, w->V, bs, Vb(j + 1), w->Hg1, sx, np);
    launch_update_gram(ctx, vprec, n, s, j + 1, w->V, bs, w->Hg1, Vb(j + 1), w->Hg2, sx, np);
    launch_update(ctx, vprec, n, s, j + 1, w->V, bs, w->Hg2, Vb(j + 1), 0, sx);
    cholqr2(ctx, vprec, n, s, Vb(j + 1), w->Rn, w->defl, sx, np);
    ProfScope psh(ctx, PF_HESS, 0.0, 4.0 * (j + 1) * s * s * (s + 1), sx);
    k_hess_old<<<s, 32, 8 * ((size_t)(j + 2) * s + (size_t)j * s * kSmallLd), sx>>>(
        j, s, ldh, w->Hg1, w->Hg2, w->Rn, w->Hb, w->refl);
    check_launch("k_hess_old");
    k_hess_step<<<1, 512, 8 * (size_t)s * (j + 2) * s, sx>>>(j, s, ldh, w->Hb, w->refl, w->Gr,
                                                            w->target, w->est, w->flag);
    check_launch("k_hess_step");
    ctx->launches += 2;
    PINT_CUDA(cudaMemcpyAsync(ctx->h_flag, w->flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, sx));
    PINT_CUDA(cudaMemcpyAsync(ctx->h_flag + 2, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                              sx));
  };
  while (res.its < o->max_inner) {
    res.cycles += 1;
    cholqr2(ctx, vprec, n, s, Vb(0), w->S, w->defl, st, np);
    {
      ProfScope ps(ctx, PF_HESS, 0.0, 0.0, st);
      k_gr_init<<<8, 256, 0, st>>>(ldh, s, w->S, w->Gr);
    }
    check_launch("k_gr_init");
    ctx->launches += 1;
    int j = 0;
    bool conv = false;
    for (j = 0; j < m; ++j) {
      arnoldi_step(j, st);
      res.its += 1;
      PINT_CUDA(cudaStreamSynchronize(st));
      PINT_REQUIRE(ctx->h_flag[2] == 0, PINT_ERR_TIMEOUT,
                   "bulk-copy wait in the Gram kernel exceeded its time budget");
      if (ilu) ilu_check(op);
      PINT_REQUIRE(ctx->h_flag[1] == 0, PINT_ERR_BREAKDOWN,
                   "non-finite residual estimate in block GMRES");
      conv = ctx->h_flag[0] != 0;
      if (conv || res.its >= o->max_inner) {
        j += 1;
        break;
      }
    }
    const int kd = j * s;
    {
      ProfScope ps(ctx, PF_HESS, 0.0, 1.0 * kd * kd * s, st);
      k_backsolve<<<1, 512, 8 * (size_t)kd * s, st>>>(kd, s, ldh, w->Hb, w->Gr, w->Yls);
      check_launch("k_backsolve");
      ctx->launches += 1;
    }
    if (ilu) {
      launch_update(ctx, vprec, n, s, j, w->V, bs, w->Yls, w->Zt, 1, st);
      void* tmp = Vb(std::min(j, m));   // block j is free after the cycle
      ilu_apply(op, prec, w->Zt, tmp, st);
      ProfScope ps(ctx, PF_VEC, 3.0 * es * ns, 1.0 * ns, st);
      if (vprec == PINT_FP64)
        k_axpy<double><<<grid_for(ns, 256), 256, 0, st>>>(ns, (const double*)tmp, (double*)w->Xk);
      else
        k_axpy<float><<<grid_for(ns, 256), 256, 0, st>>>(ns, (const float*)tmp, (float*)w->Xk);
      check_launch("k_axpy");
      ctx->launches += 1;
    } else {
      launch_update(ctx, vprec, n, s, j, w->V, bs, w->Yls, w->Xk, 2, st);
    }
    if (conv) {
      res.converged = true;
      break;
    }
    if (res.its >= o->max_inner) break;
    // restart: V_0 = Rs - J Xk
    launch_inner_spmm(op, prec, jac, w->Xk, Vb(0), w->Rs, st);
  }
  PINT_CUDA(cudaMemcpyAsync(ctx->h_flag, w->defl, sizeof(int), cudaMemcpyDeviceToHost, st));
  PINT_CUDA(cudaStreamSynchronize(st));
  res.deflations = ctx->h_flag[0];
  return res;
}

// ------------------------------------------------------ block CG (inner)
// out = scale * Rinv Rinv^T Y for the deflating Cholesky factor of G = R^T R
// (Rinv from k_chol, zero rows for deflated pivots): the inverse of a
// symmetric positive semi-definite s x s G on its active columns.
__global__ void k_spd_apply(int s, const double* __restrict__ Rinv, const double* __restrict__ Y,
                            double scale, double* __restrict__ out) {
  __shared__ double T[kMaxS][kMaxS + 1];
  const int t = threadIdx.x, i = t / kMaxS, k = t % kMaxS;
  if (i < s && k < s) {                         // T = Rinv^T Y
    double v = 0.0;
    for (int c = 0; c < s; ++c) v += Rinv[c * s + i] * Y[c * s + k];
    T[i][k] = v;
  }
  __syncthreads();
  if (i < s && k < s) {                         // out = scale Rinv T
    double v = 0.0;
    for (int c = 0; c < s; ++c) v += Rinv[i * s + c] * T[c][k];
    out[i * s + k] = scale * v;
  }
}

// Z = D^-1 R (Jacobi) in the vector precision
template <typename VT>
__global__ void k_rowscale_v(int64_t n, int s, const VT* __restrict__ R,
                             const double* __restrict__ dinv, VT* __restrict__ Z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * s) Z[i] = (VT)((double)R[i] * dinv[i / s]);
}

// Breakdown-free preconditioned block CG on the unit-column right-hand side
// Rs (symmetric positive definite J and M): the search block is
// orthonormalised by CholQR2 with deflation every iteration, so dependent or
// converged columns leave it instead of making P^T J P singular.
//   Z = M^-1 R, P = orth(Z);  repeat: Q = J P, a = (P^T Q)^+ P^T R,
//   X += P a, R -= Q a, Z = M^-1 R, b = -(P^T Q)^+ Q^T Z, P = orth(Z + P b)
// Blocks 0..3 of the basis hold P, Q, Z, R; the solution goes to Xk.
static InnerResult block_cg(pint_op op, const pint_opts* o, KrylovWork* w, cudaStream_t st) {
  pint_ctx ctx = op->ctx;
  const int64_t n = op->n;
  const int s = op->s, prec = o->precision;
  const int vprec = prec == PINT_FP64 ? PINT_FP64 : PINT_FP32;
  const bool ilu = o->precond == PINT_PC_ILU0;
  const int64_t bs = w->bs, np = w->n_pad, ns = n * s;
  const size_t es = w->es;
  PINT_REQUIRE(w->m >= 3, PINT_ERR_INVALID, "block CG needs restart >= 3 (work blocks)");
  auto Vb = [&](int b) { return (void*)((char*)w->V + (size_t)b * bs * es); };
  void* Pb = Vb(0);
  void* Qb = Vb(1);
  void* Zb = Vb(2);
  void* Rb = Vb(3);
  const double defl = vprec == PINT_FP64 ? 1e-14 : 1e-8;
  auto precond = [&](const void* X, void* Z) {
    if (ilu) {
      ilu_apply(op, prec, X, Z, st);
    } else if (o->precond == PINT_PC_JACOBI) {
      ProfScope ps(ctx, PF_VEC, (2.0 * es + 8.0) * ns, 1.0 * ns, st);
      if (vprec == PINT_FP64)
        k_rowscale_v<double><<<grid_for(ns, 256), 256, 0, st>>>(n, s, (const double*)X,
                                                                op->Jinvdiag, (double*)Z);
      else
        k_rowscale_v<float><<<grid_for(ns, 256), 256, 0, st>>>(n, s, (const float*)X,
                                                               op->Jinvdiag, (float*)Z);
      check_launch("k_rowscale_v");
      ctx->launches += 1;
    } else {
      PINT_CUDA(cudaMemcpyAsync(Z, X, es * ns, cudaMemcpyDeviceToDevice, st));
    }
  };
  auto spd_apply = [&](const double* Y, double scale, double* out) {
    ProfScope ps(ctx, PF_CHOLQR, 0.0, 4.0 * s * s * s, st);
    k_spd_apply<<<1, 256, 0, st>>>(s, w->S, Y, scale, out);
    check_launch("k_spd_apply");
    ctx->launches += 1;
  };
  {
    double t[kMaxS];
    for (int k = 0; k < s; ++k) t[k] = o->inner_tol;
    PINT_CUDA(cudaMemcpyAsync(w->target, t, 8 * s, cudaMemcpyHostToDevice, st));
  }
  PINT_CUDA(cudaMemsetAsync(w->Xk, 0, es * ns, st));
  PINT_CUDA(cudaMemsetAsync(w->defl, 0, 64, st));
  PINT_CUDA(cudaMemcpyAsync(Rb, w->Rs, es * ns, cudaMemcpyDeviceToDevice, st));
  if (s < w->s && np > n)          // narrower than the allocation: clear the padded rows
    for (int b = 0; b < 4; ++b)
      PINT_CUDA(cudaMemsetAsync((char*)Vb(b) + es * (size_t)ns, 0, es * (size_t)(np - n) * s, st));
  precond(Rb, Zb);
  PINT_CUDA(cudaMemcpyAsync(Pb, Zb, es * ns, cudaMemcpyDeviceToDevice, st));
  cholqr2(ctx, vprec, n, s, Pb, w->Rn, w->defl, st, np);
  InnerResult res{0, 1, false, 0};
  while (res.its < o->max_inner) {
    launch_inner_spmm(op, prec, false, Pb, Qb, nullptr, st);              // Q = J P
    launch_gram(ctx, vprec, n, s, 1, Pb, bs, Qb, w->Hg1, st, np);           // G = P^T Q
    {
      ProfScope ps(ctx, PF_CHOLQR, 0.0, 1.0 * s * s * s, st);
      k_chol<<<1, 256, 0, st>>>(s, w->Hg1, defl, w->Rn, w->S, w->defl);
      check_launch("k_chol");
      ctx->launches += 1;
    }
    launch_gram(ctx, vprec, n, s, 1, Pb, bs, Rb, w->Hg2, st, np);           // P^T R
    spd_apply(w->Hg2, 1.0, w->Yls);                                         // a
    launch_update(ctx, vprec, n, s, 1, Pb, bs, w->Yls, w->Xk, 2, st);       // X += P a
    launch_update(ctx, vprec, n, s, 1, Qb, bs, w->Yls, Rb, 0, st);          // R -= Q a
    launch_colnorm(ctx, vprec, n, s, Rb, w->est, st);
    res.its += 1;
    PINT_CUDA(cudaMemcpyAsync(ctx->h_small, w->est, 8 * s, cudaMemcpyDeviceToHost, st));
    PINT_CUDA(cudaMemcpyAsync(ctx->h_flag + 2, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                              st));
    PINT_CUDA(cudaStreamSynchronize(st));
    PINT_REQUIRE(ctx->h_flag[2] == 0, PINT_ERR_TIMEOUT,
                 "bulk-copy wait in the Gram kernel exceeded its time budget");
    if (ilu) ilu_check(op);
    bool conv = true;
    for (int k = 0; k < s; ++k) {
      PINT_REQUIRE(std::isfinite(ctx->h_small[k]), PINT_ERR_BREAKDOWN,
                   "non-finite residual in block CG");
      if (!(ctx->h_small[k] <= o->inner_tol)) conv = false;   // columns of Rs are unit
    }
    if (conv) {
      res.converged = true;
      break;
    }
    precond(Rb, Zb);                                                        // Z = M^-1 R
    launch_gram(ctx, vprec, n, s, 1, Qb, bs, Zb, w->Hg2, st, np);           // Q^T Z
    spd_apply(w->Hg2, -1.0, w->Yls);                                        // b
    launch_update(ctx, vprec, n, s, 1, Pb, bs, w->Yls, Zb, 2, st);          // Z += P b
    cholqr2(ctx, vprec, n, s, Zb, w->Rn, w->defl, st, np);                  // P = orth(Z)
    std::swap(Pb, Zb);
  }
  PINT_CUDA(cudaMemcpyAsync(ctx->h_flag, w->defl, sizeof(int), cudaMemcpyDeviceToHost, st));
  PINT_CUDA(cudaStreamSynchronize(st));
  res.deflations = ctx->h_flag[0];
  return res;
}

// ------------------------------------------------ block BiCGStab (inner)
// Coefficients of one block BiCGStab iteration from the Gram blocks
//   H1 = [V Rh]^T Rt (2s x s)  and  H2 = [S T Rt]^T T (3s x s):
// G = Rt^T V is the transpose of the top block of H1. Stage 0 solves
// G alpha = Rt^T Rh; stage 1 forms omega = <T, S>_F / <T, T>_F and solves
// G beta = -Rt^T T. Columns deflated at the start (zero diagonal of the
// CholQR factor C) are inactive: identity rows and columns of G, zero rows
// of the right-hand side. Gaussian elimination with partial pivoting on
// [G | rhs] in one CTA; a zero or non-finite pivot sets flag[1].
// Co holds four row-major s x s blocks: alpha, omega I, beta, -omega beta.
__global__ void __launch_bounds__(256)
k_bicg_coef(int s, int stage, const double* __restrict__ H1, const double* __restrict__ H2,
            const double* __restrict__ C, double* __restrict__ Co, int* __restrict__ flag) {
  __shared__ double A[kMaxS][2 * kMaxS + 1];
  __shared__ double mult[kMaxS];
  __shared__ int act[kMaxS];
  __shared__ double om;
  __shared__ int bad, piv;
  const int t = threadIdx.x, w2 = 2 * s;
  if (t < s) act[t] = C[t * s + t] != 0.0 ? 1 : 0;
  if (t == 0) {
    bad = 0;
    om = 0.0;
    if (stage == 1) {
      double ts = 0.0, tt = 0.0;
      for (int i = 0; i < s; ++i) {
        ts += H2[i * s + i];
        tt += H2[(s + i) * s + i];
      }
      om = tt > 0.0 ? ts / tt : 0.0;
      if (!isfinite(om)) bad = 1;
    }
  }
  __syncthreads();
  for (int e = t; e < s * w2; e += blockDim.x) {
    const int k = e / w2, c = e - k * w2;
    double v;
    if (c < s) {
      v = (act[k] && act[c]) ? H1[c * s + k] : (k == c ? 1.0 : 0.0);
    } else {
      const int j = c - s;
      v = !act[k] ? 0.0 : (stage == 0 ? H1[(s + j) * s + k] : -H2[(2 * s + k) * s + j]);
    }
    A[k][c] = v;
  }
  __syncthreads();
  for (int k = 0; k < s; ++k) {
    if (t == 0) {
      int p = k;
      double best = fabs(A[k][k]);
      for (int i = k + 1; i < s; ++i)
        if (fabs(A[i][k]) > best) {
          best = fabs(A[i][k]);
          p = i;
        }
      piv = p;
      if (!(best > 0.0) || !isfinite(best)) bad = 1;
    }
    __syncthreads();
    if (bad) break;                     // read after the barrier: uniform
    if (piv != k && t < w2) {
      const double x = A[k][t];
      A[k][t] = A[piv][t];
      A[piv][t] = x;
    }
    __syncthreads();
    if (t > k && t < s) mult[t] = A[t][k] / A[k][k];
    __syncthreads();
    const int wc = w2 - k - 1;          // columns k+1 .. 2s-1
    for (int e = t; e < (s - k - 1) * wc; e += blockDim.x) {
      const int i = k + 1 + e / wc, c = k + 1 + e % wc;
      A[i][c] -= mult[i] * A[k][c];
    }
    __syncthreads();
  }
  if (t < s && !bad) {                  // back substitution, one right-hand side per thread
    for (int k = s - 1; k >= 0; --k) {
      double v = A[k][s + t];
      for (int c = k + 1; c < s; ++c) v -= A[k][c] * A[c][s + t];
      A[k][s + t] = v / A[k][k];
    }
  }
  __syncthreads();
  if (bad && t == 0) flag[1] = 1;
  for (int e = t; e < s * s; e += blockDim.x) {
    const int i = e / s, j = e - i * s;
    const double x = bad ? 0.0 : A[i][s + j];
    if (stage == 0) {
      Co[e] = x;
    } else {
      Co[s * s + e] = i == j ? om : 0.0;
      Co[2 * s * s + e] = x;
      Co[3 * s * s + e] = -om * x;
    }
  }
}

// Block BiCGStab with right preconditioning (Guennouni, Jbilou and Sadok,
// ETNA 16, 2003) on the unit-column right-hand side Rs of a nonsymmetric J.
// Rs = Q0 C by CholQR2 with deflation, so dependent or zero columns leave the
// block before it starts; the iteration solves J Xh = Q0 with the shadow
// block Rt = Q0 and returns Xk = Xh C:
//   Rh = P = Q0;  repeat: Ph = M^-1 P, V = J Ph, alpha = (Rt^T V)^-1 Rt^T Rh,
//   S = Rh - V alpha, Sh = M^-1 S, T = J Sh, omega = <T, S>_F / <T, T>_F,
//   Xh += Ph alpha + omega Sh, Rh = S - omega T (converged when every column
//   of Rh C is <= inner_tol), beta = -(Rt^T V)^-1 Rt^T T,
//   P = Rh + (P - omega V) beta.
// With Jacobi the matrix is the column-scaled J D^-1, as in block GMRES.
// Basis blocks: 0 P, 1 V, 2 Rh (S), 3 T, 4 Rt, 5 Ph (then the new P), 6 Sh,
// 7 Xh, 8 Rh C. The runs (V, Rh), (S, T, Rt), (Ph, Sh) and (P, V) are
// adjacent, so each Gram product and block update is a single launch.
static InnerResult block_bicgstab(pint_op op, const pint_opts* o, KrylovWork* w,
                                  cudaStream_t st) {
  pint_ctx ctx = op->ctx;
  const int64_t n = op->n;
  const int s = op->s, prec = o->precision;
  const int vprec = prec == PINT_FP64 ? PINT_FP64 : PINT_FP32;
  const bool jac = o->precond == PINT_PC_JACOBI;
  const bool ilu = o->precond == PINT_PC_ILU0;
  const int64_t bs = w->bs, np = w->n_pad, ns = n * s;
  const size_t es = w->es;
  PINT_REQUIRE(w->m >= 8, PINT_ERR_INVALID, "block BiCGStab needs restart >= 8 (work blocks)");
  auto Vb = [&](int b) { return (void*)((char*)w->V + (size_t)b * bs * es); };
  void* Pb = Vb(0);
  void* Vv = Vb(1);
  void* Rh = Vb(2);
  void* Tb = Vb(3);
  void* Rt = Vb(4);
  void* Ph = Vb(5);
  void* Sh = Vb(6);
  void* Xh = Vb(7);
  void* Rc = Vb(8);
  double* Co = w->Yls;
  auto copy = [&](void* dst, const void* src) {
    PINT_CUDA(cudaMemcpyAsync(dst, src, es * ns, cudaMemcpyDeviceToDevice, st));
  };
  auto coef = [&](int stage) {
    ProfScope ps(ctx, PF_HESS, 0.0, 2.0 * s * s * s, st);
    k_bicg_coef<<<1, 256, 0, st>>>(s, stage, w->Hg1, w->Hg2, w->S, Co, w->flag);
    check_launch("k_bicg_coef");
    ctx->launches += 1;
  };
  if (s < w->s && np > n)          // narrower than the allocation: clear the padded rows
    for (int b = 0; b < 9; ++b)
      PINT_CUDA(cudaMemsetAsync((char*)Vb(b) + es * (size_t)ns, 0, es * (size_t)(np - n) * s, st));
  PINT_CUDA(cudaMemsetAsync(w->flag, 0, 64, st));
  PINT_CUDA(cudaMemsetAsync(w->defl, 0, 64, st));
  PINT_CUDA(cudaMemsetAsync(Xh, 0, es * ns, st));
  copy(Rt, w->Rs);
  cholqr2(ctx, vprec, n, s, Rt, w->S, w->defl, st, np);                     // Rs = Q0 C
  copy(Rh, Rt);
  copy(Pb, Rt);
  InnerResult res{0, 1, false, 0};
  while (res.its < o->max_inner) {
    if (ilu) ilu_apply(op, prec, Pb, Ph, st);                                // Ph = M^-1 P
    launch_inner_spmm(op, prec, jac, ilu ? Ph : Pb, Vv, nullptr, st);         // V = J Ph
    launch_gram(ctx, vprec, n, s, 2, Vv, bs, Rt, w->Hg1, st, np);             // [V Rh]^T Rt
    coef(0);                                                                  // alpha
    launch_update(ctx, vprec, n, s, 1, Vv, bs, Co, Rh, 0, st);                // S = Rh - V alpha
    if (ilu) ilu_apply(op, prec, Rh, Sh, st);                                // Sh = M^-1 S
    launch_inner_spmm(op, prec, jac, ilu ? Sh : Rh, Tb, nullptr, st);         // T = J Sh
    launch_gram(ctx, vprec, n, s, 3, Rh, bs, Tb, w->Hg2, st, np);             // [S T Rt]^T T
    coef(1);                                                                  // omega, beta
    if (ilu) {
      launch_update(ctx, vprec, n, s, 2, Ph, bs, Co, Xh, 2, st);              // Xh += [Ph Sh] [alpha; omega I]
    } else {
      launch_update(ctx, vprec, n, s, 1, Pb, bs, Co, Xh, 2, st);              // Xh += P alpha
      launch_update(ctx, vprec, n, s, 1, Rh, bs, Co + s * s, Xh, 2, st);      // Xh += omega S
    }
    launch_update(ctx, vprec, n, s, 1, Tb, bs, Co + s * s, Rh, 0, st);        // Rh = S - omega T
    launch_update(ctx, vprec, n, s, 1, Rh, bs, w->S, Rc, 1, st);              // Rh C
    launch_colnorm(ctx, vprec, n, s, Rc, w->est, st);
    res.its += 1;
    PINT_CUDA(cudaMemcpyAsync(ctx->h_small, w->est, 8 * s, cudaMemcpyDeviceToHost, st));
    PINT_CUDA(cudaMemcpyAsync(ctx->h_flag, w->flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    PINT_CUDA(cudaMemcpyAsync(ctx->h_flag + 2, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                              st));
    PINT_CUDA(cudaStreamSynchronize(st));
    PINT_REQUIRE(ctx->h_flag[2] == 0, PINT_ERR_TIMEOUT,
                 "bulk-copy wait in the Gram kernel exceeded its time budget");
    if (ilu) ilu_check(op);
    PINT_REQUIRE(ctx->h_flag[1] == 0, PINT_ERR_BREAKDOWN,
                 "singular s x s system (Rt^T V) in block BiCGStab");
    bool conv = true;
    for (int k = 0; k < s; ++k) {
      PINT_REQUIRE(std::isfinite(ctx->h_small[k]), PINT_ERR_BREAKDOWN,
                   "non-finite residual in block BiCGStab");
      if (!(ctx->h_small[k] <= o->inner_tol)) conv = false;   // columns of Rs are unit
    }
    if (conv) {
      res.converged = true;
      break;
    }
    copy(Ph, Rh);
    launch_update(ctx, vprec, n, s, 2, Pb, bs, Co + 2 * s * s, Ph, 2, st);   // Rh + [P V][beta; -omega beta]
    copy(Pb, Ph);
  }
  launch_update(ctx, vprec, n, s, 1, Xh, bs, w->S, w->Xk, 1, st);            // Xk = Xh C
  PINT_CUDA(cudaMemcpyAsync(ctx->h_flag, w->defl, sizeof(int), cudaMemcpyDeviceToHost, st));
  PINT_CUDA(cudaStreamSynchronize(st));
  res.deflations = ctx->h_flag[0];
  return res;
}

InnerResult inner_solve(pint_op op, const pint_opts* o, const double* R, const double* rnorm_dev,
                        double* /*unused*/, cudaStream_t st) {
  KrylovWork* w = ensure_work(op, o->precision == PINT_FP64 ? PINT_FP64 : PINT_FP32, o->restart);
  // the error word that bounded waits raise belongs to this solve only
  PINT_CUDA(cudaMemsetAsync(op->ctx->d_flag, 0, sizeof(int), st));
  const int64_t n = op->n;
  const int s = op->s;
  if (w->prec == PINT_FP64) {
    launch_scale_copy64(n, s, R, (double*)w->Rs, rnorm_dev, st, op->ctx);   // Rs = R / ||R_k||
  } else {
    launch_scale_cast(n, s, R, (float*)w->Rs, rnorm_dev, st, op->ctx);
  }
  if (o->solver == PINT_SOLVER_CG) return block_cg(op, o, w, st);
  if (o->solver == PINT_SOLVER_BICGSTAB) return block_bicgstab(op, o, w, st);
  return gmres(op, o, w, st);
}

void work_views(pint_op op, int prec, int m, double** R64, double** rnorm, void** Xk,
                int* wprec) {
  KrylovWork* w = ensure_work(op, prec, m);
  *R64 = w->R64;
  *rnorm = w->rnorm;
  *Xk = w->Xk;
  *wprec = w->prec;
}

// ------------------------------------------------------- outer driver
static double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------- global GMRES (unsplit operator)
// out[0] = sqrt(sum_k c[k]^2) (Frobenius norm from the column norms)
__global__ void k_frob(int s, const double* __restrict__ c, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double v = 0.0;
  for (int k = 0; k < s; ++k) v += c[k] * c[k];
  out[0] = sqrt(v);
}

// X *= 1 / nrm[0] (zero when nrm is 0)
__global__ void k_scale_by(int64_t ne, double* __restrict__ X, const double* __restrict__ nrm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ne) return;
  const double d = nrm[0];
  X[i] = d > 0.0 ? X[i] * (1.0 / d) : 0.0;
}

// Frobenius products h[b] = <V_b, W>_F of nb basis blocks with W, as per-CTA
// partials partial[cta * nb + b] over the CTA's element range (warp w takes
// the blocks w, w + 8, ...; the CTA's slice of W is read from L1 by the other
// warps), summed in a fixed order by k_gram_reduce_w.
__global__ void __launch_bounds__(256)
k_frob_dots(int64_t ne, int nb, const double* __restrict__ V, int64_t bstride,
            const double* __restrict__ W, int64_t per_cta, double* __restrict__ partial) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e0 = (int64_t)blockIdx.x * per_cta;
  const int64_t e1 = min(ne, e0 + per_cta);
  for (int b = warp; b < nb; b += 8) {
    const double* v = V + (int64_t)b * bstride;
    double acc = 0.0;
    for (int64_t e = e0 + lane; e < e1; e += 32) acc = fma(__ldg(v + e), __ldg(W + e), acc);
    acc = warp_sum(acc);
    if (lane == 0) partial[(int64_t)blockIdx.x * nb + b] = acc;
  }
}

// MODE 0: W -= sum_b h[b] V_b ; MODE 1: W = sum_b h[b] V_b (element-wise)
template <int MODE>
__global__ void __launch_bounds__(256)
k_scalar_update(int64_t ne, int nb, const double* __restrict__ V, int64_t bstride,
                const double* __restrict__ h, double* __restrict__ W) {
  __shared__ double hs[PINT_MAX_RESTART + 1];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hs[b] = h[b];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    // four blocks' loads ahead of their FMAs: 4.51 -> 4.82 TB/s in the 128^3,
    // s = 8 global GMRES solve (the same unroll slowed k_frob_dots, whose
    // warps stream their own blocks, from 2.05 to 1.48 TB/s)
#pragma unroll 4
    for (int b = 0; b < nb; ++b) acc = fma(hs[b], __ldg(V + (int64_t)b * bstride + e), acc);
    if (MODE == 0) W[e] -= acc;
    else W[e] = acc;
  }
}

// Y -= V (float64, n x s)
__global__ void k_sub(int64_t ne, const double* __restrict__ V, double* __restrict__ Y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ne) Y[i] -= V[i];
}

// Z = D^-1 X (float64 rows scaled by the inverse diagonal of J)
__global__ void k_rowscale64(int64_t n, int s, const double* __restrict__ X,
                             const double* __restrict__ dinv, double* __restrict__ Z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * s) Z[i] = X[i] * dinv[i / s];
}

// Slab solve by global GMRES(m) (Jbilou, Messaoudi and Sadok 1999) on the
// unsplit operator A(V) = M V A1^T + K V A2^T of Eq. general-system-time-steps,
// right-preconditioned column by column with the preconditioner of
// J = alpha M + beta K (P = identity, Jacobi or ILU(0)), float64. Each cycle
// solves A(V) = R(Y) from V = 0 in the Frobenius inner product
// <X, Y>_F = tr(X^T Y) and applies Y <- Y - P(V): the same defect correction
// and per-column stopping test as the split method, with the s x s coupling
// inside the Krylov space instead of in an outer fixed point. Per Arnoldi
// step: W = A(P(V_j)); two classical Gram-Schmidt passes of Frobenius
// products (k_frob_dots) and element-wise combinations (k_scalar_update);
// V_{j+1} = W / ||W||_F; the scalar Hessenberg column through the block
// kernels at width 1. A cycle ends when the least-squares
// residual estimate is below tol * min_k ||F_k|| (every column then meets its
// own tolerance) or after m steps.
static int solve_global_impl(pint_op op, const double* B, const double* B0, double* Y,
                             const pint_opts* o, pint_stats* stats, cudaStream_t st) {
  pint_ctx ctx = op->ctx;
  hist_reset(ctx, op->s);
  const double t0 = now_ms();
  const long l0 = ctx->launches;
  PINT_REQUIRE(o->precision == PINT_FP64, PINT_ERR_INVALID,
               "global GMRES runs in float64 (precision PINT_FP64)");
  const int64_t n = op->n;
  const int s = op->s, m = o->restart;
  const bool ilu = o->precond == PINT_PC_ILU0, jac = o->precond == PINT_PC_JACOBI;
  if (!op->j_valid) build_inner(op, st);
  double setup_ms = 0.0;
  if (ilu) {
    const double ts = now_ms();
    ilu_setup(op, st);
    setup_ms = now_ms() - ts;
  }
  KrylovWork* w = ensure_work(op, PINT_FP64, m);
  const int64_t bs = w->bs, np = w->n_pad, ns = n * s;
  auto Vb = [&](int b) { return (double*)w->V + (size_t)b * bs; };
  if (s < w->s && np > n)          // narrower than the allocation: clear the padded rows
    for (int b = 0; b <= m; ++b)
      PINT_CUDA(cudaMemsetAsync(Vb(b) + ns, 0, 8 * (size_t)(np - n) * s, st));
  // small state of this call: Frobenius products of the two passes, column
  // norms
  const size_t nsm = 2 * (size_t)(m + 1) + kMaxS;
  double* sm = dalloc_n<double>(ctx, nsm);
  struct Free {
    pint_ctx c;
    double* p;
    size_t b;
    ~Free() { dfree(c, p, b); }
  } fr{ctx, sm, sizeof(double) * nsm};
  double* h1 = sm;
  double* h2 = h1 + (m + 1);
  double* cn = h2 + (m + 1);
  const int ldh = m + 1;
  smem_attr(k_hess_step, 8 * (size_t)(m + 1));
  smem_attr(k_hess_old, 8 * ((size_t)(m + 1) + (size_t)m * kSmallLd));
  smem_attr(k_backsolve, 8 * (size_t)m);
  PINT_CUDA(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), st));
  auto precond = [&](const double* X, double* Z) {
    if (ilu) {
      ilu_apply(op, PINT_FP64, X, Z, st);
    } else if (jac) {
      k_rowscale64<<<grid_for(ns, 256), 256, 0, st>>>(n, s, X, op->Jinvdiag, Z);
      check_launch("k_rowscale64");
      ctx->launches += 1;
    } else {
      PINT_CUDA(cudaMemcpyAsync(Z, X, 8 * ns, cudaMemcpyDeviceToDevice, st));
    }
  };
  // Frobenius products with the first nb basis blocks (PF_GRAM) and the
  // element-wise combinations (PF_UPDATE); memory-bound, nb FMAs per element
  const int fblk = (int)std::max<int64_t>(1, std::min<int64_t>(2LL * ctx->num_sms, (ns + 2047) / 2048));
  const int64_t fper = (ns + fblk - 1) / fblk;
  ensure_partial(ctx, sizeof(double) * (size_t)fblk * (m + 1));
  auto frob_dots = [&](int nb, const double* Wd, double* h) {
    ProfScope ps(ctx, PF_GRAM, 8.0 * (nb + 1) * ns, 2.0 * nb * ns, st);
    k_frob_dots<<<fblk, 256, 0, st>>>(ns, nb, Vb(0), bs, Wd, fper, ctx->d_partial);
    check_launch("k_frob_dots");
    k_gram_reduce_launch(nb, fblk, ctx->d_partial, h, st);
    check_launch("k_gram_reduce (Frobenius)");
    ctx->launches += 2;
  };
  auto scalar_update = [&](int nb, const double* h, double* Wd, bool assign) {
    ProfScope ps(ctx, PF_UPDATE, 8.0 * (nb + (assign ? 1 : 2)) * ns, 2.0 * nb * ns, st);
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(8LL * ctx->num_sms,
                                                                       (ns + 255) / 256));
    if (assign) k_scalar_update<1><<<g, 256, 0, st>>>(ns, nb, Vb(0), bs, h, Wd);
    else k_scalar_update<0><<<g, 256, 0, st>>>(ns, nb, Vb(0), bs, h, Wd);
    check_launch("k_scalar_update");
    ctx->launches += 1;
  };
  // ||F_k|| from the residual of Y = 0
  double* Rf = w->R64;
  double* zero = (double*)w->Zt;
  PINT_CUDA(cudaMemsetAsync(zero, 0, 8 * ns, st));
  launch_coupled(op, zero, B, B0, Rf, st);
  launch_colnorm(ctx, PINT_FP64, n, s, Rf, w->fnorm, st);
  double fn[kMaxS], rn[kMaxS];
  PINT_CUDA(cudaMemcpyAsync(ctx->h_small, w->fnorm, 8 * s, cudaMemcpyDeviceToHost, st));
  PINT_CUDA(cudaStreamSynchronize(st));
  double fmin = 0.0;
  for (int k = 0; k < s; ++k) {
    fn[k] = ctx->h_small[k];
    const double thr = fn[k] > 0.0 ? o->tol * fn[k] : o->tol;
    fmin = k == 0 ? thr : std::min(fmin, thr);
  }
  PINT_CUDA(cudaMemcpyAsync(w->target, &fmin, 8, cudaMemcpyHostToDevice, st));
  int status = PINT_ERR_NOT_CONVERGED, outer = 0, inner = 0, cycles = 0;
  for (outer = 0; outer <= o->max_outer; ++outer) {
    launch_coupled(op, Y, B, B0, w->R64, st);
    launch_colnorm(ctx, PINT_FP64, n, s, w->R64, w->rnorm, st);
    PINT_CUDA(cudaMemcpyAsync(ctx->h_small, w->rnorm, 8 * s, cudaMemcpyDeviceToHost, st));
    PINT_CUDA(cudaStreamSynchronize(st));
    bool done = true, bad = false;
    for (int k = 0; k < s; ++k) {
      rn[k] = ctx->h_small[k];
      if (!std::isfinite(rn[k])) bad = true;
      if (!(rn[k] <= (fn[k] > 0.0 ? o->tol * fn[k] : o->tol))) done = false;
    }
    {
      double rel[kMaxS];
      for (int k = 0; k < s; ++k) rel[k] = fn[k] > 0.0 ? rn[k] / fn[k] : rn[k];
      hist_push(ctx, rel, s);
      if (stats)
        for (int k = 0; k < s; ++k) stats->col_relres[k] = rel[k];
    }
    if (bad) {
      status = PINT_ERR_BREAKDOWN;
      break;
    }
    if (done) {
      status = PINT_OK;
      break;
    }
    if (outer == o->max_outer || inner >= o->max_inner) break;
    cycles += 1;
    // V_0 = R / ||R||_F, right-hand side of the least squares beta e_1
    {
      ProfScope ps(ctx, PF_VEC, 16.0 * ns, 1.0 * ns, st);
      k_frob<<<1, 32, 0, st>>>(s, w->rnorm, w->S);
      PINT_CUDA(cudaMemcpyAsync(Vb(0), w->R64, 8 * ns, cudaMemcpyDeviceToDevice, st));
      k_scale_by<<<grid_for(ns, 256), 256, 0, st>>>(ns, Vb(0), w->S);
      k_gr_init<<<8, 256, 0, st>>>(ldh, 1, w->S, w->Gr);
      check_launch("global GMRES start");
      ctx->launches += 3;
    }
    int j = 0;
    bool conv = false;
    for (j = 0; j < m; ++j) {
      // W = A(P(V_j))
      if (ilu || jac) {
        precond(Vb(j), (double*)w->Zt);
        launch_coupled(op, (double*)w->Zt, nullptr, nullptr, Vb(j + 1), st);
      } else {
        launch_coupled(op, Vb(j), nullptr, nullptr, Vb(j + 1), st);
      }
      // two classical Gram-Schmidt passes in the Frobenius inner product
      for (int pass = 0; pass < 2; ++pass) {
        double* hp = pass == 0 ? h1 : h2;
        frob_dots(j + 1, Vb(j + 1), hp);
        scalar_update(j + 1, hp, Vb(j + 1), false);
      }
      // V_{j+1} = W / ||W||_F, then the Hessenberg column (h1 + h2; ||W||_F)
      launch_colnorm(ctx, PINT_FP64, n, s, Vb(j + 1), cn, st);
      {
        ProfScope ps(ctx, PF_HESS, 0.0, 4.0 * (j + 2), st);
        k_frob<<<1, 32, 0, st>>>(s, cn, w->Rn);
        k_scale_by<<<grid_for(ns, 256), 256, 0, st>>>(ns, Vb(j + 1), w->Rn);
        k_hess_old<<<1, 32, 8 * ((size_t)(j + 2) + (size_t)j * kSmallLd), st>>>(
            j, 1, ldh, h1, h2, w->Rn, w->Hb, w->refl);
        k_hess_step<<<1, 512, 8 * (size_t)(j + 2), st>>>(j, 1, ldh, w->Hb, w->refl, w->Gr,
                                                         w->target, w->est, w->flag);
        check_launch("global GMRES Hessenberg");
        ctx->launches += 4;
      }
      PINT_CUDA(cudaMemcpyAsync(ctx->h_flag, w->flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
      PINT_CUDA(cudaMemcpyAsync(ctx->h_flag + 2, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                                st));
      PINT_CUDA(cudaStreamSynchronize(st));
      inner += 1;
      PINT_REQUIRE(ctx->h_flag[2] == 0, PINT_ERR_TIMEOUT,
                   "bulk-copy wait in the Gram kernel exceeded its time budget");
      if (ilu) ilu_check(op);
      PINT_REQUIRE(ctx->h_flag[1] == 0, PINT_ERR_BREAKDOWN,
                   "non-finite residual estimate in global GMRES");
      conv = ctx->h_flag[0] != 0;
      if (conv || inner >= o->max_inner) {
        j += 1;
        break;
      }
    }
    // correction V = P(sum_b y_b V_b), Y <- Y - V
    const int kd = std::min(j, m);
    {
      ProfScope ps(ctx, PF_HESS, 0.0, 1.0 * kd * kd, st);
      k_backsolve<<<1, 512, 8 * (size_t)kd, st>>>(kd, 1, ldh, w->Hb, w->Gr, w->Yls);
      check_launch("k_backsolve");
      ctx->launches += 1;
    }
    scalar_update(kd, w->Yls, (double*)w->Zt, true);
    double* corr = Vb(kd);                       // free after the cycle
    precond((const double*)w->Zt, corr);
    {
      ProfScope ps(ctx, PF_VEC, 24.0 * ns, 1.0 * ns, st);
      k_sub<<<grid_for(ns, 256), 256, 0, st>>>(ns, corr, Y);
      check_launch("k_sub");
      ctx->launches += 1;
    }
  }
  PINT_CUDA(cudaStreamSynchronize(st));
  if (stats) {
    stats->status = status;
    stats->outer_its = outer;
    stats->inner_its = inner;
    stats->restarts = cycles;
    stats->deflations = 0;
    stats->setup_ms = setup_ms;
    stats->solve_ms = now_ms() - t0;
    stats->kernel_launches = (int)(ctx->launches - l0);
  }
  if (status == PINT_ERR_BREAKDOWN) throw Error{PINT_ERR_BREAKDOWN, "non-finite outer residual"};
  return status;
}

int solve_block_impl(pint_op op, const double* B, const double* B0, double* Y,
                     const pint_opts* o, pint_stats* stats, cudaStream_t st) {
  pint_ctx ctx = op->ctx;
  hist_reset(ctx, op->s);
  const double t0 = now_ms();
  const long l0 = ctx->launches;
  PINT_REQUIRE(op->s >= 1, PINT_ERR_INVALID, "coupling not set (pint_set_coupling)");
  PINT_REQUIRE(o->restart >= 1 && o->restart <= PINT_MAX_RESTART, PINT_ERR_INVALID,
               "restart out of range");
  PINT_REQUIRE((int64_t)(o->restart + 1) * op->s <= 1024, PINT_ERR_INVALID,
               "(restart + 1) * s must not exceed 1024");
  PINT_REQUIRE(8 * ((size_t)op->s * (o->restart + 1) * op->s +
                    (size_t)o->restart * op->s * kSmallLd) <= 227 * 1024,
               PINT_ERR_INVALID, "restart too long for this block width (Hessenberg shared memory)");
  PINT_REQUIRE(o->precision >= PINT_FP64 && o->precision <= PINT_BF16, PINT_ERR_INVALID,
               "precision");
  PINT_REQUIRE(o->precond >= PINT_PC_NONE && o->precond <= PINT_PC_ILU0, PINT_ERR_INVALID,
               "precond");
  PINT_REQUIRE(o->solver >= PINT_SOLVER_GMRES && o->solver <= PINT_SOLVER_GLOBAL,
               PINT_ERR_INVALID, "solver");
  if (o->solver == PINT_SOLVER_GLOBAL) return solve_global_impl(op, B, B0, Y, o, stats, st);
  const int64_t n = op->n;
  const int s = op->s;
  if (!op->j_valid) build_inner(op, st);
  double setup_ms = 0.0;
  if (o->precond == PINT_PC_ILU0) {
    const double ts = now_ms();
    ilu_setup(op, st);
    setup_ms = now_ms() - ts;
  }
  KrylovWork* w = ensure_work(op, o->precision == PINT_FP64 ? PINT_FP64 : PINT_FP32, o->restart);
  // ||F_k|| with F = B A2^T + B0: residual of Y = 0 is -F
  PINT_CUDA(cudaMemsetAsync(w->Zt, 0, w->es * (size_t)n * s, st));
  double* zeroY = nullptr;
  if (w->es == 8) {
    zeroY = (double*)w->Zt;
  } else {
    zeroY = (double*)w->V;   // first 8*n*s bytes of the basis are free here
    PINT_CUDA(cudaMemsetAsync(zeroY, 0, 8 * (size_t)n * s, st));
  }
  launch_coupled(op, zeroY, B, B0, w->R64, st);
  launch_colnorm(ctx, PINT_FP64, n, s, w->R64, w->fnorm, st);
  double fn[kMaxS], rn[kMaxS];
  PINT_CUDA(cudaMemcpyAsync(ctx->h_small, w->fnorm, 8 * s, cudaMemcpyDeviceToHost, st));
  PINT_CUDA(cudaStreamSynchronize(st));
  for (int k = 0; k < s; ++k) fn[k] = ctx->h_small[k];
  bool lower = true;                 // both coupling matrices lower triangular
  for (int i = 0; i < s; ++i)
    for (int k = i + 1; k < s; ++k)
      if (op->A1[i * kMaxS + k] != 0.0 || op->A2[i * kMaxS + k] != 0.0) lower = false;
  int status = PINT_ERR_NOT_CONVERGED;
  int outer = 0, inner = 0, cycles = 0, defl = 0;
  for (outer = 0; outer <= o->max_outer; ++outer) {
    launch_coupled(op, Y, B, B0, w->R64, st);
    launch_colnorm(ctx, PINT_FP64, n, s, w->R64, w->rnorm, st);
    PINT_CUDA(cudaMemcpyAsync(ctx->h_small, w->rnorm, 8 * s, cudaMemcpyDeviceToHost, st));
    PINT_CUDA(cudaStreamSynchronize(st));
    bool done = true, bad = false;
    for (int k = 0; k < s; ++k) {
      rn[k] = ctx->h_small[k];
      if (!std::isfinite(rn[k])) bad = true;
      const double thr = fn[k] > 0.0 ? o->tol * fn[k] : o->tol;
      if (!(rn[k] <= thr)) done = false;
    }
    {
      double rel[kMaxS];
      for (int k = 0; k < s; ++k) rel[k] = fn[k] > 0.0 ? rn[k] / fn[k] : rn[k];
      hist_push(ctx, rel, s);
      if (stats)
        for (int k = 0; k < s; ++k) stats->col_relres[k] = rel[k];
    }
    if (bad) {
      status = PINT_ERR_BREAKDOWN;
      break;
    }
    if (done) {
      status = PINT_OK;
      break;
    }
    if (outer == o->max_outer) break;
    // With lower-triangular A1, A2 the residual of column k depends on
    // columns 0..k of Y only, so a converged leading run of columns stays
    // converged: the inner solve is narrowed to the trailing columns
    // (power-of-two width, so that the kernels keep their exact-width forms;
    // the few converged columns it still carries are harmless).
    int c0 = 0;
    if (lower) {
      int lead = 0;
      while (lead < s && rn[lead] <= (fn[lead] > 0.0 ? o->tol * fn[lead] : o->tol)) ++lead;
      int wdt = 1;
      while (wdt < s - lead) wdt <<= 1;
      if (wdt < s) c0 = s - wdt;
    }
    const int sw = s - c0;
    InnerResult ir;
    if (c0 == 0) {
      ir = inner_solve(op, o, w->R64, w->rnorm, nullptr, st);
    } else {
      launch_gather_cols(n, s, c0, sw, w->R64, w->Rsub, st, ctx);
      struct WidthGuard {
        pint_op op;
        int s0;
        ~WidthGuard() { op->s = s0; }
      } guard{op, s};
      op->s = sw;
      ir = inner_solve(op, o, w->Rsub, w->rnorm + c0, nullptr, st);
    }
    inner += ir.its;
    cycles += ir.cycles;
    defl += ir.deflations;
    const int vprec = w->prec;
    // block GMRES and block BiCGStab with Jacobi solve for the scaled
    // variable D X (right preconditioning fused into the SpMM); block CG
    // solves for X itself
    const bool scaled = o->precond == PINT_PC_JACOBI && o->solver != PINT_SOLVER_CG;
    launch_outer_update(vprec, n, sw, Y, w->Xk, w->rnorm + c0, scaled ? op->Jinvdiag : nullptr,
                        st, ctx, s, c0);
  }
  PINT_CUDA(cudaStreamSynchronize(st));
  if (stats) {
    stats->status = status;
    stats->outer_its = outer;
    stats->inner_its = inner;
    stats->restarts = cycles;
    stats->deflations = defl;
    stats->setup_ms = setup_ms;
    stats->solve_ms = now_ms() - t0;
    stats->kernel_launches = (int)(ctx->launches - l0);
  }
  if (status == PINT_ERR_BREAKDOWN)
    throw Error{PINT_ERR_BREAKDOWN, "non-finite outer residual"};
  return status;
}

}  // namespace pint

// ===================================================================
// Block Gram product without any device allocation.
//
// pint_block_gram needs a context, and the context allocates device memory
// (cudaMalloc) for its reduction buffers. Some callers cannot allow that: code
// that runs inside a framework whose caching allocator already owns the
// device memory pool, real-time loops that must never allocate, and paths that
// must not take the implicit device synchronisation of cudaMalloc/cudaFree.
// pint_block_gram_noalloc computes the same H = [V_1..V_nb]^T W with the
// cross-CTA partial sums kept in the file-scope device array below instead.
// ===================================================================
namespace pint {

// 4 MiB of float64 partial sums, resident on every device that loads the
// library until the process exits.
constexpr int kNoAllocScratchDoubles = 1 << 19;
constexpr int kNoAllocMaxBlocks = 128;      // CTAs of the Gram launch
constexpr int kNoAllocMaxEntries = kNoAllocScratchDoubles / kNoAllocMaxBlocks;   // nb*s*s
static __device__ __align__(256) double g_gram_scratch[kNoAllocScratchDoubles];

struct NoAllocDevice {
  bool ready = false;
  double* scratch = nullptr;   // device address of g_gram_scratch on this device
  int num_sms = 0;
};
static NoAllocDevice g_noalloc_dev[64];
static std::mutex g_noalloc_mutex;

void set_noctx_error(const std::string& msg);   // api.cu

template <typename VT>
static void gram_noalloc_t(const NoAllocDevice& d, int64_t n, int s, int nb, const VT* V,
                           const VT* W, double* H, cudaStream_t st) {
  const int P = nb * s;
  int PT = 32;
  while (PT < P && PT < 256) PT <<= 1;
  const int npt = (P + PT - 1) / PT;
  const int64_t want = std::max<int64_t>(
      1, std::min<int64_t>(std::min(4 * d.num_sms, kNoAllocMaxBlocks), (n + 63) / 64));
  int64_t rpc = (n + want - 1) / want;
  rpc = std::max<int64_t>(kGramTile, ((rpc + kGramTile - 1) / kGramTile) * kGramTile);
  const int nblk = (int)((n + rpc - 1) / rpc);
  const int E = P * s;
  const size_t tile_bytes = sizeof(VT) * kGramTile * (P + s);
  const size_t red_bytes = sizeof(double) * E;
  const size_t smem = std::max(tile_bytes, (PT < 256 ? red_bytes : (size_t)0));
  with_s(s, [&](auto S_, auto E_) {
    constexpr int S = decltype(S_)::value;
    constexpr bool EX = decltype(E_)::value;
    auto launch = [&](auto kern) {
      smem_attr(kern, smem);
      kern<<<nblk, 256, smem, st>>>(n, s, nb, V, n * s, W, rpc, d.scratch);
    };
    if (npt == 1) launch(k_gram<VT, S, EX, 1>);
    else if (npt == 2) launch(k_gram<VT, S, EX, 2>);
    else launch(k_gram<VT, S, EX, 4>);
  });
  check_launch("k_gram (no-alloc)");
  k_gram_reduce<<<(E + 255) / 256, 256, 0, st>>>(nblk, E, d.scratch, H);
  check_launch("k_gram_reduce (no-alloc)");
}

}  // namespace pint

extern "C" int pint_block_gram_noalloc(int precision, int64_t n, int s, int nb, const void* V,
                                       const void* W, double* H, void* stream) {
  using namespace pint;
  try {
    PINT_REQUIRE(n >= 1 && s >= 1 && s <= PINT_MAX_S && nb >= 1, PINT_ERR_INVALID,
                 "pint_block_gram_noalloc: need n >= 1, 1 <= s <= 16, nb >= 1");
    PINT_REQUIRE((int64_t)nb * s * s <= kNoAllocMaxEntries, PINT_ERR_INVALID,
                 "pint_block_gram_noalloc: nb*s*s = " + std::to_string((int64_t)nb * s * s) +
                     " exceeds the maximum of " + std::to_string(kNoAllocMaxEntries) +
                     " (fixed scratch of 4 MiB)");
    // the Gram kernel covers at most 4 x 256 basis columns per CTA
    PINT_REQUIRE((int64_t)nb * s <= 1024, PINT_ERR_INVALID,
                 "pint_block_gram_noalloc: nb*s = " + std::to_string((int64_t)nb * s) +
                     " exceeds the maximum of 1024 basis columns");
    PINT_REQUIRE(precision == PINT_FP64 || precision == PINT_FP32, PINT_ERR_INVALID,
                 "pint_block_gram_noalloc: precision must be PINT_FP64 or PINT_FP32");
    PINT_REQUIRE(V && W && H, PINT_ERR_INVALID, "pint_block_gram_noalloc: NULL pointer");
    PINT_REQUIRE(reinterpret_cast<uintptr_t>(V) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(W) % 16 == 0,
                 PINT_ERR_INVALID, "pint_block_gram_noalloc: V and W must be 16-byte aligned");
    int dev = 0;
    PINT_CUDA(cudaGetDevice(&dev));
    PINT_REQUIRE(dev >= 0 && dev < 64, PINT_ERR_INVALID, "pint_block_gram_noalloc: device index");
    NoAllocDevice d;
    {
      std::lock_guard<std::mutex> lk(g_noalloc_mutex);
      NoAllocDevice& slot = g_noalloc_dev[dev];
      if (!slot.ready) {   // once per device, with that device current
        void* p = nullptr;
        PINT_CUDA(cudaGetSymbolAddress(&p, g_gram_scratch));
        PINT_CUDA(cudaDeviceGetAttribute(&slot.num_sms, cudaDevAttrMultiProcessorCount, dev));
        slot.scratch = static_cast<double*>(p);
        slot.ready = true;
      }
      d = slot;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (precision == PINT_FP64)
      gram_noalloc_t<double>(d, n, s, nb, (const double*)V, (const double*)W, H, st);
    else
      gram_noalloc_t<float>(d, n, s, nb, (const float*)V, (const float*)W, H, st);
    return PINT_OK;
  } catch (const Error& e) {
    set_noctx_error(e.msg);
    return e.code;
  }
}
