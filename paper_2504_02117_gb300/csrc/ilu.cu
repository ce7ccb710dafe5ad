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
  // row-of-tiles sweeps (stencil operators): tile shape, row order, flags,
  // stencil-format factors L4 / U4 ([n][4], float64 and float32)
  bool rows = false;
  int RX = 0, RY = 0, RZ = 0, RNTX = 0, RNTY = 0, RNTZ = 0, rntiles = 0, nrows = 0;
  int* row_order = nullptr;
  unsigned* rflag_f = nullptr;
  unsigned* rflag_b = nullptr;
  unsigned repoch_f = 0, repoch_b = 0;
  double* L4d = nullptr;
  double* U4d = nullptr;
  float* L4f = nullptr;
  float* U4f = nullptr;
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

// 16-byte asynchronous global -> shared copy (L2 only) and its groups
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src_gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst_smem)),
               "l"(src_gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
// all committed groups but the most recent one have completed
__device__ __forceinline__ void cp_async_wait_prev() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

// Wait until flag == epoch. Returns false (and raises *err) when the budget
// is exhausted, or at once when another thread has raised *err.
__device__ __forceinline__ bool wait_ready(const unsigned* flag, unsigned epoch, int* err,
                                           unsigned long long deadline) {
  if (ld_acquire(flag) == epoch) return true;
  for (unsigned it = 1;; ++it) {
    if ((it & 63) == 0) {
      if (*(volatile int*)err != 0) return false;
      if (globaltimer() > deadline) {
        atomicExch(err, 1);
        return false;
      }
    }
    __nanosleep(20);
    if (ld_acquire(flag) == epoch) return true;
  }
}

// Test of the bounded dependency wait: one thread waits through wait_ready
// for `flag` to reach epoch 1, which nothing stores, with a deadline
// `budget_ns` from now; it raises *err (1) and returns.
__global__ void k_test_wait_timeout(const unsigned* flag, unsigned long long budget_ns, int* err) {
  if (threadIdx.x == 0) wait_ready(flag, 1u, err, globaltimer() + budget_ns);
}

void test_wait_timeout(double limit_ms, unsigned* flag, int* err, cudaStream_t st) {
  k_test_wait_timeout<<<1, 32, 0, st>>>(flag, (unsigned long long)(limit_ms * 1e6), err);
  check_launch("k_test_wait_timeout");
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

// ------------------------------------------------ stencil (grid) sweeps
// For the natural-order 7-point (5-point in 2-D) stencil, row (i,j,k) reads
// only (i-1,j,k), (i,j-1,k), (i,j,k-1) forward and the +1 neighbours
// backward; the sweeps below work on tiles of the grid.
struct TileGeom {
  int nx, ny, nz, NTX, NTY, ntiles;
};

// Stencil-format copy of the factors: per row four coefficients,
// FWD (L): (-z, -y, -x, 0); BWD (U): (+x, +y, +z, 1/diag); absent
// neighbours 0. The reciprocal (rounded once, in float64) turns the
// backward sweep's division into a multiplication.
template <typename VT>
__global__ void k_ilu_stencil_coefs(TileGeom g, int64_t n, const int* __restrict__ rowptr,
                                    const int* __restrict__ diagpos, const double* __restrict__ F,
                                    VT* __restrict__ L4, VT* __restrict__ U4) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int i = (int)(r % g.nx), j = (int)((r / g.nx) % g.ny), k = (int)(r / ((int64_t)g.nx * g.ny));
  double l[3] = {0, 0, 0}, u[4] = {0, 0, 0, 0};
  int p = rowptr[r];
  if (k > 0) l[0] = F[p++];
  if (j > 0) l[1] = F[p++];
  if (i > 0) l[2] = F[p++];
  const int d = diagpos[r];
  p = d + 1;
  if (i + 1 < g.nx) u[0] = F[p++];
  if (j + 1 < g.ny) u[1] = F[p++];
  if (k + 1 < g.nz) u[2] = F[p++];
  u[3] = 1.0 / F[d];
  for (int q = 0; q < 3; ++q) L4[4 * r + q] = (VT)l[q];
  L4[4 * r + 3] = VT(0);
  for (int q = 0; q < 4; ++q) U4[4 * r + q] = (VT)u[q];
}

// Row-of-tiles sweep: a CTA takes one x-row of tiles (fixed J, K; tickets
// in order of J + K, so it only waits for rows with lower tickets) and
// sweeps its tiles along x. The x-neighbour of a tile's first cells is the
// last cell of the previous tile of the same row, carried in a register; the
// y- and z-neighbours come from the rows (J-1, K) and (J, K-1) through one
// flag per tile (bounded waits). Inside a tile, thread (c, lj, lk) owns the
// x-pencil of column c and step t of the local wavefront handles its cell
// li = t - lj - lk (mirrored backward); values and coefficients are staged
// in shared memory. Same operands and order of operations per cell as the
// CSR sweep.
template <typename VT, bool FWD, int TX, int TY, int TZ, int MAXT>
__global__ void __launch_bounds__(MAXT)
k_ilu_rows(TileGeom g, int s, const VT* __restrict__ C4, const VT* X, VT* Z,
           const int* __restrict__ row_order, int nrows, unsigned* tflags, unsigned epoch,
           int* ticket, int* err) {
  constexpr int NSTEP = TX + TY + TZ - 2;
  constexpr int TR = TX * TY * TZ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  VT* Ys = reinterpret_cast<VT*>(smem_raw);        // [lk][lj][li][c]
  VT* Cb = Ys + (size_t)TR * s;                     // 2 x [lk][lj][li][4]
  VT* Hy = Cb + (size_t)2 * TR * 4;                 // [lk][li][c]
  VT* Hz = Hy + (size_t)TZ * TX * s;                // [lj][li][c]
  __shared__ int row_sh;
  const int c = threadIdx.x % s;
  const int q = threadIdx.x / s;
  const int lj = q % TY, lk = q / TY;
  const unsigned long long deadline = globaltimer() + kWaitBudgetNs;
  const int64_t sxy = (int64_t)g.nx * g.ny;
  const int NTZ = (g.nz + TZ - 1) / TZ;
  bool ok = true;
  // this pencil's right-hand side for one tile, loaded into registers with
  // all loads in flight together (unrolled, guarded)
  VT xv[TX];
  auto fetch = [&](int x0, int ex, int64_t lbase, bool mine) {
#pragma unroll
    for (int li = 0; li < TX; ++li) {
      if (mine && li < ex) {
        const int64_t r = lbase + li;
        xv[li] = FWD ? X[r * s + c] : __ldcg(Z + r * s + c);
      }
    }
  };
  // the tile's coefficients: asynchronous 16-byte copies straight into one
  // of two shared buffers, one commit group per tile
  auto fetch_coefs = [&](int I, int y0, int z0, int ey, int ez, VT* dst) {
    const int x0 = I * TX, ex = min(TX, g.nx - x0);
    constexpr int CH = 4 * (int)sizeof(VT) / 16;     // 16-byte chunks per cell
    for (int e = threadIdx.x; e < TR * CH; e += blockDim.x) {
      const int cell = e / CH, part = e - cell * CH;
      const int li = cell % TX, qq = cell / TX, ljj = qq % TY, lkk = qq / TY;
      if (li < ex && ljj < ey && lkk < ez) {
        const int64_t r = x0 + li + (int64_t)g.nx * (y0 + ljj) + sxy * (z0 + lkk);
        cp_async16(dst + (size_t)cell * 4 + part * (16 / sizeof(VT)),
                   C4 + 4 * r + part * (16 / sizeof(VT)));
      }
    }
    cp_async_commit();
  };
  while (true) {
    if (threadIdx.x == 0) {
      const int t = atomicAdd(ticket, 1);
      row_sh = t < nrows ? row_order[FWD ? t : nrows - 1 - t] : -1;
    }
    __syncthreads();
    const int row = row_sh;
    if (row < 0) return;
    const int J = row % g.NTY, K = row / g.NTY;
    const int y0 = J * TY, z0 = K * TZ;
    const int ey = min(TY, g.ny - y0), ez = min(TZ, g.nz - z0);
    const bool mine = lj < ey && lk < ez;
    const int gj = y0 + lj, gk = z0 + lk;
    const int cellb = (lk * TY + lj) * TX;
    VT hx = VT(0);                                   // carried x-neighbour
    {
      const int I = FWD ? 0 : g.NTX - 1;
      const int x0 = I * TX;
      fetch(x0, min(TX, g.nx - x0), x0 + (int64_t)g.nx * gj + sxy * gk, mine);
      fetch_coefs(I, y0, z0, ey, ez, Cb);
    }
    for (int it = 0; it < g.NTX; ++it) {
      const int I = FWD ? it : g.NTX - 1 - it;
      const int x0 = I * TX;
      const int ex = min(TX, g.nx - x0);
      const int tile = I + g.NTX * (J + g.NTY * K);
      const int64_t lbase = x0 + (int64_t)g.nx * gj + sxy * gk;   // row of li = 0
      const VT* Cs = Cb + (size_t)(it & 1) * TR * 4;
      // stage the prefetched pencil into shared memory
      if (mine) {
#pragma unroll
        for (int li = 0; li < TX; ++li)
          if (li < ex) Ys[(cellb + li) * s + c] = xv[li];
      }
      // prefetch the next tile of the row now: its loads are in flight while
      // this tile waits, computes and publishes
      if (it + 1 < g.NTX) {
        const int In = FWD ? it + 1 : g.NTX - 2 - it;
        const int xn = In * TX;
        fetch(xn, min(TX, g.nx - xn), xn + (int64_t)g.nx * gj + sxy * gk, mine);
        fetch_coefs(In, y0, z0, ey, ez, Cb + (size_t)((it + 1) & 1) * TR * 4);
      } else {
        cp_async_commit();                         // keep one group per tile
      }
      cp_async_wait_prev();                        // this tile's coefficients have landed
      // upstream rows: FWD (J-1, K), (J, K-1); BWD (J+1, K), (J, K+1)
      if (threadIdx.x < 2 && ok) {
        int nt = -1;
        if (FWD) {
          if (threadIdx.x == 0 && J > 0) nt = tile - g.NTX;
          if (threadIdx.x == 1 && K > 0) nt = tile - g.NTX * g.NTY;
        } else {
          if (threadIdx.x == 0 && J + 1 < g.NTY) nt = tile + g.NTX;
          if (threadIdx.x == 1 && K + 1 < NTZ) nt = tile + g.NTX * g.NTY;
        }
        if (nt >= 0) ok = wait_ready(tflags + nt, epoch, err, deadline);
      }
      __syncthreads();
      // faces of the y / z upstream rows (zero where the grid ends)
      if (mine) {
        const bool ybnd = FWD ? lj == 0 : lj == ey - 1;
        const bool zbnd = FWD ? lk == 0 : lk == ez - 1;
        const int64_t yoff = FWD ? -(int64_t)g.nx : (int64_t)g.nx;
        const int64_t zoff = FWD ? -sxy : sxy;
        const bool yin = FWD ? gj > 0 : gj + 1 < g.ny;
        const bool zin = FWD ? gk > 0 : gk + 1 < g.nz;
        VT hyv[TX], hzv[TX];
#pragma unroll
        for (int li = 0; li < TX; ++li) {
          hyv[li] = (ybnd && yin && li < ex) ? __ldcg(Z + (lbase + li + yoff) * s + c) : VT(0);
          hzv[li] = (zbnd && zin && li < ex) ? __ldcg(Z + (lbase + li + zoff) * s + c) : VT(0);
        }
#pragma unroll
        for (int li = 0; li < TX; ++li) {
          if (ybnd) Hy[(lk * TX + li) * s + c] = hyv[li];
          if (zbnd) Hz[(lj * TX + li) * s + c] = hzv[li];
        }
      }
      __syncthreads();
      for (int t = 0; t < NSTEP; ++t) {
        const int li = FWD ? t - lj - lk : (ex - 1) - (t - (ey - 1 - lj) - (ez - 1 - lk));
        if (mine && li >= 0 && li < ex) {
          const int cell = cellb + li;
          VT acc = Ys[cell * s + c];
          const VT* cf = Cs + cell * 4;
          if (FWD) {
            const VT vz = lk > 0 ? Ys[(cell - TY * TX) * s + c] : Hz[(lj * TX + li) * s + c];
            const VT vy = lj > 0 ? Ys[(cell - TX) * s + c] : Hy[(lk * TX + li) * s + c];
            const VT vx = li > 0 ? Ys[(cell - 1) * s + c] : hx;
            acc -= cf[0] * vz;
            acc -= cf[1] * vy;
            acc -= cf[2] * vx;
          } else {
            const VT vx = li + 1 < ex ? Ys[(cell + 1) * s + c] : hx;
            const VT vy = lj + 1 < ey ? Ys[(cell + TX) * s + c] : Hy[(lk * TX + li) * s + c];
            const VT vz = lk + 1 < ez ? Ys[(cell + TY * TX) * s + c] : Hz[(lj * TX + li) * s + c];
            acc -= cf[0] * vx;
            acc -= cf[1] * vy;
            acc -= cf[2] * vz;
            acc *= cf[3];
          }
          Ys[cell * s + c] = acc;
        }
        __syncthreads();
      }
      // Publish first what the downstream rows read: the pencils of the
      // last y row and the last z layer of the tile (FWD; the first ones
      // BWD). The release then waits only for those stores; the interior
      // stores and the next tile's loads are issued after it.
      const bool face = mine && (FWD ? ((lj == ey - 1 && J + 1 < g.NTY) || (lk == ez - 1 && K + 1 < NTZ))
                                     : ((lj == 0 && J > 0) || (lk == 0 && K > 0)));
      VT zv[TX];
      if (mine) {
        hx = Ys[(cellb + (FWD ? ex - 1 : 0)) * s + c];
#pragma unroll
        for (int li = 0; li < TX; ++li) zv[li] = li < ex ? Ys[(cellb + li) * s + c] : VT(0);
      }
      if (face) {
#pragma unroll
        for (int li = 0; li < TX; ++li)
          if (li < ex) Z[(lbase + li) * s + c] = zv[li];
      }
      // every face store of the CTA precedes thread 0's release store in
      // causality order through the barrier (which also ends all reads of
      // Ys): the barrier synchronises the storing threads with thread 0, and
      // a gpu-scope release is cumulative, so the downstream CTA that
      // acquires the flag reads the faces without a separate fence (a
      // __threadfence before the release cost 6.5 % of the 128^3 s = 8
      // float32 apply, 684 -> 640 us, with bitwise equal results)
      __syncthreads();
      if (threadIdx.x == 0) st_release(tflags + tile, epoch);
      if (mine && !face) {
#pragma unroll
        for (int li = 0; li < TX; ++li)
          if (li < ex) Z[(lbase + li) * s + c] = zv[li];
      }
    }
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

static unsigned next_epoch(pint_op op, unsigned& e, unsigned* flags, cudaStream_t st,
                           int64_t count = -1) {
  if (e >= 0xFFFFFF00u) {
    PINT_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned) * (count < 0 ? op->n : count), st));
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
  if (op->grid_nx > 0) {
    const int nx = op->grid_nx, ny = op->grid_ny, nz = op->grid_nz;
    // row-of-tiles structures
    S->RX = nz > 1 ? 8 : (ny > 1 ? 16 : 64);
    S->RY = nz > 1 ? 8 : (ny > 1 ? 8 : 1);
    S->RZ = nz > 1 ? 8 : 1;
    S->RNTX = (nx + S->RX - 1) / S->RX;
    S->RNTY = (ny + S->RY - 1) / S->RY;
    S->RNTZ = (nz + S->RZ - 1) / S->RZ;
    S->rntiles = S->RNTX * S->RNTY * S->RNTZ;
    S->nrows = S->RNTY * S->RNTZ;
    std::vector<int> ro(S->nrows);
    for (int r = 0; r < S->nrows; ++r) ro[r] = r;
    std::stable_sort(ro.begin(), ro.end(), [&](int a, int b) {
      return a % S->RNTY + a / S->RNTY < b % S->RNTY + b / S->RNTY;
    });
    S->row_order = dalloc_n<int>(ctx, S->nrows);
    S->rflag_f = dalloc_n<unsigned>(ctx, S->rntiles);
    S->rflag_b = dalloc_n<unsigned>(ctx, S->rntiles);
    S->L4d = dalloc_n<double>(ctx, 4 * op->n);
    S->U4d = dalloc_n<double>(ctx, 4 * op->n);
    S->L4f = dalloc_n<float>(ctx, 4 * op->n);
    S->U4f = dalloc_n<float>(ctx, 4 * op->n);
    PINT_CUDA(cudaMemcpy(S->row_order, ro.data(), sizeof(int) * S->nrows, cudaMemcpyHostToDevice));
    PINT_CUDA(cudaMemset(S->rflag_f, 0, sizeof(unsigned) * S->rntiles));
    PINT_CUDA(cudaMemset(S->rflag_b, 0, sizeof(unsigned) * S->rntiles));
    S->rows = true;
  }
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
  if (S->rows) {
    dfree(c, S->row_order, sizeof(int) * S->nrows);
    dfree(c, S->rflag_f, sizeof(unsigned) * S->rntiles);
    dfree(c, S->rflag_b, sizeof(unsigned) * S->rntiles);
    dfree(c, S->L4d, sizeof(double) * 4 * op->n);
    dfree(c, S->U4d, sizeof(double) * 4 * op->n);
    dfree(c, S->L4f, sizeof(float) * 4 * op->n);
    dfree(c, S->U4f, sizeof(float) * 4 * op->n);
  }
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
  if (S->rows) {
    TileGeom g{op->grid_nx, op->grid_ny, op->grid_nz, 0, 0, 0};
    k_ilu_stencil_coefs<double><<<grid_for(op->n, 256), 256, 0, st>>>(
        g, op->n, op->rowptr, op->diagpos, S->F64, S->L4d, S->U4d);
    k_ilu_stencil_coefs<float><<<grid_for(op->n, 256), 256, 0, st>>>(
        g, op->n, op->rowptr, op->diagpos, S->F64, S->L4f, S->U4f);
    check_launch("k_ilu_stencil_coefs");
    op->ctx->launches += 2;
  }
  PINT_CUDA(cudaStreamSynchronize(st));
  ilu_check(op);
  S->factored = true;
}

// shared memory of k_ilu_rows: the tile (s values per cell), two coefficient
// tiles and the y / z halos
template <typename VT>
static size_t rows_smem(int TX, int TY, int TZ, int s) {
  const size_t TR = (size_t)TX * TY * TZ;
  return sizeof(VT) * (TR * s + 2 * TR * 4 + (size_t)TZ * TX * s + (size_t)TY * TX * s);
}

template <typename VT, int TX, int TY, int TZ, int MAXT>
static void rows_pair(pint_op op, const VT* L4, const VT* U4, const VT* X, VT* Z,
                      cudaStream_t st) {
  IluState* S = op->ilu;
  const int s = op->s;
  const int NTX = (op->grid_nx + TX - 1) / TX;      // TX == S->RX
  TileGeom g{op->grid_nx, op->grid_ny, op->grid_nz, NTX, S->RNTY, NTX * S->RNTY * S->RNTZ};
  const int threads = TY * TZ * s;
  const size_t smem = rows_smem<VT>(TX, TY, TZ, s);
  const unsigned ef = next_epoch(op, S->repoch_f, S->rflag_f, st, S->rntiles);
  const unsigned eb = next_epoch(op, S->repoch_b, S->rflag_b, st, S->rntiles);
  PINT_CUDA(cudaMemsetAsync(S->ticket, 0, 2 * sizeof(int), st));
  ProfScope ps(op->ctx, PF_ILU,
               8.0 * sizeof(VT) * op->n + 4.0 * sizeof(VT) * op->n * s, 2.0 * op->nnz * s, st);
  auto launch = [&](auto kern, const VT* C, const VT* x, unsigned* flags, unsigned ep, int* tk) {
    smem_attr(kern, smem);
    int per_sm = 0;
    PINT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    const int grid = std::max(1, std::min(S->nrows, std::max(1, per_sm) * op->ctx->num_sms));
    kern<<<grid, threads, smem, st>>>(g, s, C, x, Z, S->row_order, S->nrows, flags, ep, tk,
                                      S->err);
  };
  launch(k_ilu_rows<VT, true, TX, TY, TZ, MAXT>, L4, X, S->rflag_f, ef, S->ticket);
  check_launch("k_ilu_rows<fwd>");
  launch(k_ilu_rows<VT, false, TX, TY, TZ, MAXT>, U4, Z, S->rflag_b, eb, S->ticket + 1);
  check_launch("k_ilu_rows<bwd>");
  op->ctx->launches += 2;
}

template <typename VT>
static void apply_rows(pint_op op, const VT* L4, const VT* U4, const VT* X, VT* Z,
                       cudaStream_t st) {
  IluState* S = op->ilu;
  if (S->RZ == 8 && op->s <= 8) rows_pair<VT, 8, 8, 8, 512>(op, L4, U4, X, Z, st);
  else if (S->RZ == 8) rows_pair<VT, 8, 8, 8, 1024>(op, L4, U4, X, Z, st);
  else if (S->RY == 8) rows_pair<VT, 16, 8, 1, 128>(op, L4, U4, X, Z, st);
  else rows_pair<VT, 64, 1, 1, 16>(op, L4, U4, X, Z, st);
}

template <typename VT>
static void apply_t(pint_op op, const VT* F, const VT* X, VT* Z, cudaStream_t st) {
  IluState* S = op->ilu;
  if (S->rows && op->s * S->RY * S->RZ <= 1024 &&
      rows_smem<VT>(S->RX, S->RY, S->RZ, op->s) <= 227 * 1024) {
    if constexpr (sizeof(VT) == 8) apply_rows<double>(op, S->L4d, S->U4d, X, Z, st);
    else apply_rows<float>(op, S->L4f, S->U4f, X, Z, st);
    return;
  }
  const int s = op->s;
  int spl = 0;
  while ((1 << spl) < s) ++spl;
  const int rpw = 32 >> spl;
  Sched& f = schedule(op, true, rpw);
  Sched& b = schedule(op, false, rpw);
  const unsigned ef = next_epoch(op, S->epoch_f, S->flag_f, st);
  const unsigned eb = next_epoch(op, S->epoch_b, S->flag_b, st);
  ProfScope ps(op->ctx, PF_ILU,
               op->nnz * (sizeof(VT) + 4.0) + 4.0 * (op->n + 1) + 8.0 * op->n + 8.0 * op->n +
                   4.0 * sizeof(VT) * op->n * s,
               2.0 * op->nnz * s, st);
  PINT_CUDA(cudaMemsetAsync(S->ticket, 0, 2 * sizeof(int), st));
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
