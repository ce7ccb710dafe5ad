// Sparse block kernels: SELL-32 build, the fused coupled residual (Sec. 2.2
// residual / Eq. matrix-fixed-point-equation), the inner operator apply
// J X = (alpha M + beta K) X (Sec. 3, BOP kernel), column norms, casts and
// the outer update. One thread owns one row and its s accumulators (the s
// "SIMD lanes" of Sec. 3 become registers); a warp owns one SELL slice, so
// matrix values and column indices are read once per s columns, coalesced.
#include "internal.h"

#include <algorithm>

namespace pint {

// ---------------------------------------------------------------- SELL build
void sell_build(pint_op op) {
  const int64_t n = op->n;
  const int64_t ns = (n + kSellC - 1) / kSellC;
  std::vector<int64_t> sptr(ns + 1, 0);
  for (int64_t q = 0; q < ns; ++q) {
    int w = 0;
    for (int64_t r = q * kSellC; r < std::min<int64_t>(n, (q + 1) * kSellC); ++r)
      w = std::max(w, op->h_rowptr[r + 1] - op->h_rowptr[r]);
    sptr[q + 1] = sptr[q] + (int64_t)w * kSellC;
  }
  const int64_t ne = sptr[ns];
  std::vector<int> col(ne);
  std::vector<int64_t> map(op->nnz);
  for (int64_t q = 0; q < ns; ++q) {
    const int w = (int)((sptr[q + 1] - sptr[q]) / kSellC);
    for (int l = 0; l < kSellC; ++l) {
      const int64_t r = q * kSellC + l;
      for (int t = 0; t < w; ++t) {
        const int64_t pos = sptr[q] + (int64_t)t * kSellC + l;
        if (r < n && op->h_rowptr[r] + t < op->h_rowptr[r + 1]) {
          const int64_t p = op->h_rowptr[r] + t;
          col[pos] = op->h_colind[p];
          map[p] = pos;
        } else {
          col[pos] = (int)std::min<int64_t>(r, n - 1);   // padding: own row, value 0
        }
      }
    }
  }
  SellPattern& S = op->sell;
  S.n = n;
  S.nslices = ns;
  S.nelem = ne;
  S.slice_ptr = dalloc_n<int64_t>(op->ctx, ns + 1);
  S.col = dalloc_n<int>(op->ctx, std::max<int64_t>(ne, 1));
  S.csr_to_sell = dalloc_n<int64_t>(op->ctx, std::max<int64_t>(op->nnz, 1));
  PINT_CUDA(cudaMemcpy(S.slice_ptr, sptr.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice));
  PINT_CUDA(cudaMemcpy(S.col, col.data(), sizeof(int) * ne, cudaMemcpyHostToDevice));
  PINT_CUDA(cudaMemcpy(S.csr_to_sell, map.data(), sizeof(int64_t) * op->nnz, cudaMemcpyHostToDevice));
}

template <typename OT>
__global__ void k_sell_scatter(int64_t nnz, const int* __restrict__ rowptr_unused,
                               const int64_t* __restrict__ map, const double* __restrict__ src,
                               const int* __restrict__ colind, const double* __restrict__ colscale,
                               OT* __restrict__ dst) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  double v = src[p];
  if (colscale) v *= colscale[colind[p]];
  if constexpr (std::is_same<OT, double>::value) dst[map[p]] = v;
  else if constexpr (std::is_same<OT, float>::value) dst[map[p]] = __double2float_rn(v);
  else dst[map[p]] = __double2bfloat16(v);
}

void sell_scatter(pint_op op, const double* csr_vals, double* sell_vals, cudaStream_t st) {
  if (sell_vals == op->sellK) op->stenK_valid = false;   // K's values change
  PINT_CUDA(cudaMemsetAsync(sell_vals, 0, sizeof(double) * op->sell.nelem, st));
  k_sell_scatter<double><<<grid_for(op->nnz, 256), 256, 0, st>>>(
      op->nnz, nullptr, op->sell.csr_to_sell, csr_vals, op->colind, nullptr, sell_vals);
  check_launch("k_sell_scatter");
  op->ctx->launches += 1;
}

// ------------------------------------------------ inner operator J values
__global__ void k_build_inner(int64_t n, const int* __restrict__ rowptr,
                              const int* __restrict__ diagpos, const double* __restrict__ K,
                              const double* __restrict__ M, double alpha, double beta,
                              double* __restrict__ J, double* __restrict__ Jd,
                              double* __restrict__ Jinv) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) J[p] = beta * K[p];
  const int d = diagpos[r];
  J[d] += alpha * (M ? M[r] : 1.0);
  Jd[r] = J[d];
  Jinv[r] = 1.0 / J[d];
}

void build_inner(pint_op op, cudaStream_t st) {
  if (!op->Jval) {
    op->Jval = dalloc_n<double>(op->ctx, op->nnz);
    op->Jdiag = dalloc_n<double>(op->ctx, op->n);
    op->Jinvdiag = dalloc_n<double>(op->ctx, op->n);
  }
  k_build_inner<<<grid_for(op->n, 256), 256, 0, st>>>(op->n, op->rowptr, op->diagpos, op->Kval,
                                                      op->Mdiag, op->alpha, op->beta, op->Jval,
                                                      op->Jdiag, op->Jinvdiag);
  check_launch("k_build_inner");
  op->ctx->launches += 1;
  op->j_valid = true;
}

void* inner_sell(pint_op op, int precision, bool jacobi, cudaStream_t st) {
  void*& slot = op->sellJ[precision][jacobi ? 1 : 0];
  if (slot) return slot;
  const size_t es = precision == PINT_FP64 ? 8 : precision == PINT_FP32 ? 4 : 2;
  slot = dalloc(op->ctx, es * op->sell.nelem);
  PINT_CUDA(cudaMemsetAsync(slot, 0, es * op->sell.nelem, st));
  const double* cs = jacobi ? op->Jinvdiag : nullptr;
  const unsigned g = grid_for(op->nnz, 256);
  if (precision == PINT_FP64)
    k_sell_scatter<double><<<g, 256, 0, st>>>(op->nnz, nullptr, op->sell.csr_to_sell, op->Jval,
                                              op->colind, cs, static_cast<double*>(slot));
  else if (precision == PINT_FP32)
    k_sell_scatter<float><<<g, 256, 0, st>>>(op->nnz, nullptr, op->sell.csr_to_sell, op->Jval,
                                             op->colind, cs, static_cast<float*>(slot));
  else
    k_sell_scatter<__nv_bfloat16><<<g, 256, 0, st>>>(op->nnz, nullptr, op->sell.csr_to_sell,
                                                     op->Jval, op->colind, cs,
                                                     static_cast<__nv_bfloat16*>(slot));
  check_launch("k_sell_scatter(J)");
  op->ctx->launches += 1;
  return slot;
}

// Stencil copy of a grid operator's CSR values (layout: see the inner SpMM).
template <typename OT>
__global__ void k_stencil_coefs(int64_t n, int nx, int ny, int nz, const int* __restrict__ rowptr,
                                const double* __restrict__ vals,
                                const double* __restrict__ colscale, OT* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t sxy = (int64_t)nx * ny;
  const int i = (int)(r % nx), j = (int)((r / nx) % ny), k = (int)(r / sxy);
  const int64_t nb[7] = {r - sxy, r - nx, r - 1, r, r + 1, r + nx, r + sxy};
  const bool has[7] = {k > 0, j > 0, i > 0, true, i + 1 < nx, j + 1 < ny, k + 1 < nz};
  int p = rowptr[r];
  for (int q = 0; q < 8; ++q) {
    double v = 0.0;
    if (q < 7 && has[q]) {
      v = vals[p++];
      if (colscale) v *= colscale[nb[q]];
    }
    if constexpr (std::is_same<OT, double>::value) out[8 * r + q] = v;
    else if constexpr (std::is_same<OT, float>::value) out[8 * r + q] = __double2float_rn(v);
    else out[8 * r + q] = __double2bfloat16(v);
  }
}

// --------------------------------------------------- fused coupled residual
// R_r = d_r (Y_r A1^T) + ((K Y)_r - B_r) A2^T - B0_r  for every row r, with the
// s x s products unrolled against the kernel-parameter copies of A1, A2.
// LO > 0: both matrices are lower banded with band LO (entries only at
// 0 <= i - k <= LO, the shape of the time-stepping matrices), so only that band
// is unrolled; LO == 0: dense, zero coefficients skipped by uniform branches.
// STEN: K in the stencil form of the grid operators (8 coefficients per row in
// CSR order, see the inner SpMM below): the seven rows of Y are loaded at once
// and accumulated in the same order as the SELL form.
template <int S, bool EXACT, int LO, bool STEN>
__global__ void __launch_bounds__(256)
k_coupled(int64_t n, int s, const int64_t* __restrict__ sptr, const int* __restrict__ col,
          const double* __restrict__ val, const double* __restrict__ Md,
          const double* __restrict__ Y, const double* __restrict__ B,
          const double* __restrict__ B0, double* __restrict__ R,
          const __grid_constant__ Coupling cp, int nx, int64_t sxy) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  double ky[S];
#pragma unroll
  for (int k = 0; k < S; ++k) ky[k] = 0.0;
  if constexpr (STEN) {
    double c[8];
    const double2* cq = reinterpret_cast<const double2*>(val + 8 * row);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double2 v = __ldg(cq + i);
      c[2 * i] = v.x; c[2 * i + 1] = v.y;
    }
    const int64_t off[7] = {-sxy, -(int64_t)nx, -1, 0, 1, nx, sxy};
    double x[7][S];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const int64_t nb = row + off[q];
      load_row<S, EXACT>(Y + ((nb >= 0 && nb < n) ? nb : row) * s, s, x[q]);
    }
#pragma unroll
    for (int q = 0; q < 7; ++q)
#pragma unroll
      for (int k = 0; k < S; ++k) ky[k] = fma(c[q], x[q][k], ky[k]);
  } else {
    const int64_t q = row >> 5;
    const int lane = (int)(row & 31);
    const int64_t b0 = sptr[q];
    const int w = (int)((sptr[q + 1] - b0) >> 5);
    const double* vp = val + b0 + lane;
    const int* cpp = col + b0 + lane;
    for (int t = 0; t < w; ++t) {
      const double v = __ldg(vp + (int64_t)t * 32);
      const int c = __ldg(cpp + (int64_t)t * 32);
      if (!PINT_INDEX_OK(c, n, 1)) continue;
      double x[S];
      load_row<S, EXACT>(Y + (int64_t)c * s, s, x);
#pragma unroll
      for (int k = 0; k < S; ++k) ky[k] = fma(v, x[k], ky[k]);
    }
  }
  double y[S], bb[S], out[S];
  load_row<S, EXACT>(Y + row * s, s, y);
  if (B) {
    load_row<S, EXACT>(B + row * s, s, bb);
#pragma unroll
    for (int k = 0; k < S; ++k) ky[k] -= bb[k];
  }
  if (B0) {
    load_row<S, EXACT>(B0 + row * s, s, out);
#pragma unroll
    for (int k = 0; k < S; ++k) out[k] = -out[k];
  } else {
#pragma unroll
    for (int k = 0; k < S; ++k) out[k] = 0.0;
  }
  const double d = Md ? __ldg(Md + row) : 1.0;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    if (!EXACT && i >= s) break;
    double m1 = 0.0, m2 = 0.0;
#pragma unroll
    for (int k = 0; k < S; ++k) {
      if (!EXACT && k >= s) break;
      if (LO > 0 && (k > i || i - k > LO)) continue;
      const double a1 = cp.A1[i * kMaxS + k];
      const double a2 = cp.A2[i * kMaxS + k];
      if (LO > 0) {
        m1 = fma(a1, y[k], m1);
        m2 = fma(a2, ky[k], m2);
      } else {
        if (a1 != 0.0) m1 = fma(a1, y[k], m1);
        if (a2 != 0.0) m2 = fma(a2, ky[k], m2);
      }
    }
    out[i] += fma(d, m1, m2);
  }
  store_row<S, EXACT>(R + row * s, s, out);
}

// Lower band width LO (1 or 2) when every non-zero of A1 and A2 sits at
// 0 <= i - k <= LO, else 0 (dense).
int coupling_band(const double* A1, const double* A2, int s) {
  int lo = 0;
  for (int i = 0; i < s; ++i)
    for (int k = 0; k < s; ++k)
      if (A1[i * kMaxS + k] != 0.0 || A2[i * kMaxS + k] != 0.0) {
        if (k > i) return 0;
        lo = std::max(lo, i - k);
      }
  if (lo > 2) return 0;
  return std::max(lo, 1);
}

void launch_coupled(pint_op op, const double* Y, const double* B, const double* B0, double* R,
                    cudaStream_t st) {
  Coupling cp;
  std::copy(op->A1, op->A1 + kMaxS * kMaxS, cp.A1);
  std::copy(op->A2, op->A2 + kMaxS * kMaxS, cp.A2);
  const int s = op->s;
  int nza = 0;
  for (int i = 0; i < s; ++i)
    for (int k = 0; k < s; ++k) nza += (op->A1[i * kMaxS + k] != 0.0) + (op->A2[i * kMaxS + k] != 0.0);
  const double N = (double)op->n;
  ProfScope ps(op->ctx, PF_COUPLED,
               op->nnz * 12.0 + 4.0 * (N + 1) + (op->Mdiag ? 8.0 * N : 0.0) +
                   8.0 * N * s * (2 + (B ? 1 : 0) + (B0 ? 1 : 0)),
               2.0 * op->nnz * s + 2.0 * N * nza, st);
  const int lo = coupling_band(op->A1, op->A2, s);
  const bool sten = op->grid_nx > 0;
  if (sten && !op->stenK_valid) {
    if (!op->stenK) op->stenK = dalloc_n<double>(op->ctx, 8 * op->n);
    k_stencil_coefs<double><<<grid_for(op->n, 256), 256, 0, st>>>(
        op->n, op->grid_nx, op->grid_ny, op->grid_nz, op->rowptr, op->Kval, nullptr, op->stenK);
    check_launch("k_stencil_coefs(K)");
    op->ctx->launches += 1;
    op->stenK_valid = true;
  }
  const int nx = op->grid_nx;
  const int64_t sxy = (int64_t)op->grid_nx * op->grid_ny;
  with_s(s, [&](auto S_, auto E_) {
    constexpr int S = decltype(S_)::value;
    constexpr bool E = decltype(E_)::value;
    auto launch = [&](auto kern) {
      kern<<<grid_for(op->n, 256), 256, 0, st>>>(op->n, s, op->sell.slice_ptr, op->sell.col,
                                                 sten ? op->stenK : op->sellK, op->Mdiag, Y, B,
                                                 B0, R, cp, nx, sxy);
    };
    if (sten) {
      if (lo == 1) launch(k_coupled<S, E, 1, true>);
      else if (lo == 2) launch(k_coupled<S, E, 2, true>);
      else launch(k_coupled<S, E, 0, true>);
    } else {
      if (lo == 1) launch(k_coupled<S, E, 1, false>);
      else if (lo == 2) launch(k_coupled<S, E, 2, false>);
      else launch(k_coupled<S, E, 0, false>);
    }
  });
  check_launch("k_coupled");
  op->ctx->launches += 1;
}

// ------------------------------------------------------- inner SpMM (a4)
// MODE 0: Z = J X ; MODE 1: Z = Rin - J X
template <typename MT, typename VT, int S, bool EXACT, int MODE>
__global__ void __launch_bounds__(256)
k_spmm(int64_t n, int s, const int64_t* __restrict__ sptr, const int* __restrict__ col,
       const MT* __restrict__ val, const VT* __restrict__ X, VT* __restrict__ Z,
       const VT* __restrict__ Rin) {
  using A = VT;
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const int64_t q = row >> 5;
  const int lane = (int)(row & 31);
  const int64_t b0 = sptr[q];
  const int w = (int)((sptr[q + 1] - b0) >> 5);
  A acc[S];
#pragma unroll
  for (int k = 0; k < S; ++k) acc[k] = A(0);
  const MT* vp = val + b0 + lane;
  const int* cpp = col + b0 + lane;
  for (int t = 0; t < w; ++t) {
    const A v = to_acc(vp[(int64_t)t * 32], A(0));
    const int c = __ldg(cpp + (int64_t)t * 32);
    if (!PINT_INDEX_OK(c, n, 2)) continue;
    A x[S];
    load_row<S, EXACT>(X + (int64_t)c * s, s, x);
#pragma unroll
    for (int k = 0; k < S; ++k) acc[k] = fma(v, x[k], acc[k]);
  }
  if constexpr (MODE == 1) {
    A r[S];
    load_row<S, EXACT>(Rin + row * s, s, r);
#pragma unroll
    for (int k = 0; k < S; ++k) acc[k] = r[k] - acc[k];
  }
  store_row<S, EXACT>(Z + row * s, s, acc);
}

// ------------------------------------- inner SpMM, stencil form (a4)
// Operators of the FV constructors have the natural-order 7-point pattern
// (5-point in 2-D, 3-point in 1-D): row r holds at most the entries of the
// columns r - nx ny, r - nx, r - 1, r, r + 1, r + nx, r + nx ny, in this
// (CSR) order. The stencil copy keeps them 8 to a row in that order (absent
// neighbours 0, slot 7 padding), so one row's coefficients are one aligned
// 16- or 32-byte load and the neighbour rows of X are read at fixed offsets
// by consecutive threads: coalesced, without column indices. The products are
// accumulated in the same order as the CSR / SELL form, so both forms give
// the same result.
void* inner_stencil(pint_op op, int precision, bool jacobi, cudaStream_t st) {
  void*& slot = op->stenJ[precision][jacobi ? 1 : 0];
  if (slot) return slot;
  const size_t es = precision == PINT_FP64 ? 8 : precision == PINT_FP32 ? 4 : 2;
  slot = dalloc(op->ctx, es * 8 * op->n);
  const double* cs = jacobi ? op->Jinvdiag : nullptr;
  const unsigned g = grid_for(op->n, 256);
  const int nx = op->grid_nx, ny = op->grid_ny, nz = op->grid_nz;
  if (precision == PINT_FP64)
    k_stencil_coefs<double><<<g, 256, 0, st>>>(op->n, nx, ny, nz, op->rowptr, op->Jval, cs,
                                               static_cast<double*>(slot));
  else if (precision == PINT_FP32)
    k_stencil_coefs<float><<<g, 256, 0, st>>>(op->n, nx, ny, nz, op->rowptr, op->Jval, cs,
                                              static_cast<float*>(slot));
  else
    k_stencil_coefs<__nv_bfloat16><<<g, 256, 0, st>>>(op->n, nx, ny, nz, op->rowptr, op->Jval,
                                                      cs, static_cast<__nv_bfloat16*>(slot));
  check_launch("k_stencil_coefs");
  op->ctx->launches += 1;
  return slot;
}

// the 8 stencil coefficients of one row, as the accumulation type
template <typename MT, typename A>
__device__ __forceinline__ void ld_coef8(const MT* __restrict__ p, A (&c)[8]) {
  if constexpr (std::is_same<MT, double>::value) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double2 v = __ldg(q + i);
      c[2 * i] = v.x; c[2 * i + 1] = v.y;
    }
  } else if constexpr (std::is_same<MT, float>::value) {
    const float4* q = reinterpret_cast<const float4*>(p);
    const float4 a = __ldg(q), b = __ldg(q + 1);
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
  } else {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __bfloat1622float2(h[i]);
      c[2 * i] = f.x; c[2 * i + 1] = f.y;
    }
  }
}

// MODE 0: Z = J X ; MODE 1: Z = Rin - J X
// Row mapping: TILED (grids with ny > 1) gives a block of 32 x 8 threads a
// patch of 32 x-cells by 8 y-lines of one z-plane (grid nx/32 x ny/8 x nz), so
// most +-1 and +-nx neighbour rows are rows the same block reads; otherwise
// 256 consecutive rows.
template <typename MT, typename VT, int S, bool EXACT, int MODE, bool TILED>
__global__ void __launch_bounds__(256)
k_stencil(int64_t n, int nx, int ny, int s, const MT* __restrict__ C8,
          const VT* __restrict__ X, VT* __restrict__ Z, const VT* __restrict__ Rin) {
  using A = VT;
  const int64_t sxy = (int64_t)nx * ny;
  int64_t row;
  if constexpr (TILED) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    if (i >= nx || j >= ny) return;
    row = i + (int64_t)nx * j + sxy * blockIdx.z;
  } else {
    row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
  }
  A c[8];
  ld_coef8<MT, A>(C8 + 8 * row, c);
  // all seven rows are loaded at once (an absent neighbour, whose coefficient
  // is 0, reads the row itself), then accumulated in the CSR order
  const int64_t off[7] = {-sxy, -(int64_t)nx, -1, 0, 1, nx, sxy};
  A x[7][S];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const int64_t nb = row + off[q];
    load_row<S, EXACT>(X + ((nb >= 0 && nb < n) ? nb : row) * s, s, x[q]);
  }
  A acc[S];
#pragma unroll
  for (int k = 0; k < S; ++k) acc[k] = A(0);
#pragma unroll
  for (int q = 0; q < 7; ++q)
#pragma unroll
    for (int k = 0; k < S; ++k) acc[k] = fma(c[q], x[q][k], acc[k]);
  if constexpr (MODE == 1) {
    A r[S];
    load_row<S, EXACT>(Rin + row * s, s, r);
#pragma unroll
    for (int k = 0; k < S; ++k) acc[k] = r[k] - acc[k];
  }
  store_row<S, EXACT>(Z + row * s, s, acc);
}

static void launch_stencil_spmm(pint_op op, int precision, bool jacobi, const void* X, void* Z,
                                const void* Rin, cudaStream_t st) {
  void* val = inner_stencil(op, precision, jacobi, st);
  const int s = op->s;
  const unsigned g = grid_for(op->n, 256);
  const double vs = precision == PINT_FP64 ? 8.0 : precision == PINT_FP32 ? 4.0 : 2.0;
  const double xs = precision == PINT_FP64 ? 8.0 : 4.0;
  // algorithmic bytes of the product in CSR form (values and int32 column
  // indices of the nnz entries, the row pointer, X read and Z written once,
  // Rin read once), the same count as the SELL form books; the stencil form
  // itself moves 8 coefficients per row instead of the nnz values and indices
  ProfScope ps(op->ctx, PF_SPMM,
               op->nnz * (vs + 4.0) + 4.0 * (op->n + 1) + xs * op->n * s * (Rin ? 3 : 2),
               2.0 * op->nnz * s, st);
  const int nx = op->grid_nx, ny = op->grid_ny, nz = op->grid_nz;
  const bool tiled = ny > 1;
  const dim3 tb(32, 8);
  const dim3 tg((unsigned)((nx + 31) / 32), (unsigned)((ny + 7) / 8), (unsigned)nz);
  with_s(s, [&](auto S_, auto E_) {
    constexpr int S = decltype(S_)::value;
    constexpr bool E = decltype(E_)::value;
    auto go = [&](auto kflat, auto ktile, const auto* v, const auto* x, auto* z, const auto* rin) {
      if (tiled) ktile<<<tg, tb, 0, st>>>(op->n, nx, ny, s, v, x, z, rin);
      else kflat<<<g, 256, 0, st>>>(op->n, nx, ny, s, v, x, z, rin);
    };
    if (precision == PINT_FP64) {
      if (Rin) go(k_stencil<double, double, S, E, 1, false>, k_stencil<double, double, S, E, 1, true>, (const double*)val, (const double*)X,
                  (double*)Z, (const double*)Rin);
      else go(k_stencil<double, double, S, E, 0, false>, k_stencil<double, double, S, E, 0, true>, (const double*)val, (const double*)X,
              (double*)Z, (const double*)nullptr);
    } else if (precision == PINT_FP32) {
      if (Rin) go(k_stencil<float, float, S, E, 1, false>, k_stencil<float, float, S, E, 1, true>, (const float*)val, (const float*)X,
                  (float*)Z, (const float*)Rin);
      else go(k_stencil<float, float, S, E, 0, false>, k_stencil<float, float, S, E, 0, true>, (const float*)val, (const float*)X, (float*)Z,
              (const float*)nullptr);
    } else {
      if (Rin) go(k_stencil<__nv_bfloat16, float, S, E, 1, false>, k_stencil<__nv_bfloat16, float, S, E, 1, true>, (const __nv_bfloat16*)val,
                  (const float*)X, (float*)Z, (const float*)Rin);
      else go(k_stencil<__nv_bfloat16, float, S, E, 0, false>, k_stencil<__nv_bfloat16, float, S, E, 0, true>, (const __nv_bfloat16*)val,
              (const float*)X, (float*)Z, (const float*)nullptr);
    }
  });
  check_launch("k_stencil");
  op->ctx->launches += 1;
}

void launch_inner_spmm(pint_op op, int precision, bool jacobi, const void* X, void* Z,
                       const void* Rin, cudaStream_t st) {
  if (op->grid_nx > 0) {
    launch_stencil_spmm(op, precision, jacobi, X, Z, Rin, st);
    return;
  }
  void* val = inner_sell(op, precision, jacobi, st);
  const int s = op->s;
  const unsigned g = grid_for(op->n, 256);
  const double vs = precision == PINT_FP64 ? 8.0 : precision == PINT_FP32 ? 4.0 : 2.0;
  const double xs = precision == PINT_FP64 ? 8.0 : 4.0;
  ProfScope ps(op->ctx, PF_SPMM,
               op->nnz * (vs + 4.0) + 4.0 * (op->n + 1) + xs * op->n * s * (Rin ? 3 : 2),
               2.0 * op->nnz * s, st);
  with_s(s, [&](auto S_, auto E_) {
    constexpr int S = decltype(S_)::value;
    constexpr bool E = decltype(E_)::value;
    auto& P = op->sell;
    if (precision == PINT_FP64) {
      if (Rin)
        k_spmm<double, double, S, E, 1><<<g, 256, 0, st>>>(
            op->n, s, P.slice_ptr, P.col, (const double*)val, (const double*)X, (double*)Z,
            (const double*)Rin);
      else
        k_spmm<double, double, S, E, 0><<<g, 256, 0, st>>>(
            op->n, s, P.slice_ptr, P.col, (const double*)val, (const double*)X, (double*)Z,
            nullptr);
    } else if (precision == PINT_FP32) {
      if (Rin)
        k_spmm<float, float, S, E, 1><<<g, 256, 0, st>>>(
            op->n, s, P.slice_ptr, P.col, (const float*)val, (const float*)X, (float*)Z,
            (const float*)Rin);
      else
        k_spmm<float, float, S, E, 0><<<g, 256, 0, st>>>(
            op->n, s, P.slice_ptr, P.col, (const float*)val, (const float*)X, (float*)Z, nullptr);
    } else {
      if (Rin)
        k_spmm<__nv_bfloat16, float, S, E, 1><<<g, 256, 0, st>>>(
            op->n, s, P.slice_ptr, P.col, (const __nv_bfloat16*)val, (const float*)X, (float*)Z,
            (const float*)Rin);
      else
        k_spmm<__nv_bfloat16, float, S, E, 0><<<g, 256, 0, st>>>(
            op->n, s, P.slice_ptr, P.col, (const __nv_bfloat16*)val, (const float*)X, (float*)Z,
            nullptr);
    }
  });
  check_launch("k_spmm");
  op->ctx->launches += 1;
}

// ---------------------------------------------------------- column norms
constexpr int kNormBlocks = 512;

template <typename VT, int S, bool EXACT>
__global__ void __launch_bounds__(256)
k_colsq(int64_t n, int s, const VT* __restrict__ X, double* __restrict__ partial) {
  double acc[S];
#pragma unroll
  for (int k = 0; k < S; ++k) acc[k] = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    VT x[S];
    load_row<S, EXACT>(X + r * s, s, x);
#pragma unroll
    for (int k = 0; k < S; ++k) acc[k] = fma((double)x[k], (double)x[k], acc[k]);
  }
  __shared__ double red[8][S];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    double v = warp_sum(acc[k]);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < S) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
    partial[blockIdx.x * kMaxS + threadIdx.x] = v;
  }
}

// one warp per column, fixed summation order (deterministic)
__global__ void k_colsq_final(int nblk, int s, const double* __restrict__ partial,
                              double* __restrict__ out) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= s) return;
  double v = 0.0;
#pragma unroll 4
  for (int b = lane; b < nblk; b += 32) v += partial[b * kMaxS + k];
  v = warp_sum(v);
  if (lane == 0) out[k] = sqrt(v);
}

void launch_colnorm(pint_ctx ctx, int precision, int64_t n, int s, const void* X, double* out,
                    cudaStream_t st) {
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kNormBlocks, (n + 255) / 256));
  double* partial = ctx->d_small + kSmallNormPartial;
  ProfScope ps(ctx, PF_NORM, (precision == PINT_FP64 ? 8.0 : 4.0) * n * s, 2.0 * n * s, st);
  with_s(s, [&](auto S_, auto E_) {
    constexpr int S = decltype(S_)::value;
    constexpr bool E = decltype(E_)::value;
    if (precision == PINT_FP64)
      k_colsq<double, S, E><<<nb, 256, 0, st>>>(n, s, (const double*)X, partial);
    else
      k_colsq<float, S, E><<<nb, 256, 0, st>>>(n, s, (const float*)X, partial);
  });
  k_colsq_final<<<1, 32 * kMaxS, 0, st>>>(nb, s, partial, out);
  check_launch("k_colsq");
  ctx->launches += 2;
}

// ---------------------------------------------------- outer update (a10)
// Y[r][yoff + k] -= colscale[k] * rowscale[r] * V[r][k]  (V: n x s, Y: n x ys)
template <typename VT>
__global__ void k_outer_update(int64_t n, int s, double* __restrict__ Y, int ys, int yoff,
                               const VT* __restrict__ V, const double* __restrict__ colscale,
                               const double* __restrict__ rowscale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * s) return;
  const int64_t r = i / s;
  const int k = (int)(i - r * s);
  double v = (double)V[i] * colscale[k];
  if (rowscale) v *= rowscale[r];
  Y[r * ys + yoff + k] -= v;
}

void launch_outer_update(int precision, int64_t n, int s, double* Y, const void* V,
                         const double* colscale, const double* rowscale, cudaStream_t st,
                         pint_ctx ctx, int ys, int yoff) {
  const unsigned g = grid_for(n * s, 256);
  if (ys <= 0) ys = s;
  ProfScope ps(ctx, PF_VEC, (16.0 + (precision == PINT_FP64 ? 8.0 : 4.0)) * n * s +
                                (rowscale ? 8.0 * n : 0.0), 3.0 * n * s, st);
  if (precision == PINT_FP64)
    k_outer_update<double><<<g, 256, 0, st>>>(n, s, Y, ys, yoff, (const double*)V, colscale,
                                              rowscale);
  else
    k_outer_update<float><<<g, 256, 0, st>>>(n, s, Y, ys, yoff, (const float*)V, colscale,
                                             rowscale);
  check_launch("k_outer_update");
  ctx->launches += 1;
}

// dst (n x w) = columns c0 .. c0 + w - 1 of src (n x s), float64
__global__ void k_gather_cols(int64_t n, int s, int c0, int w, const double* __restrict__ src,
                              double* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * w) return;
  const int64_t r = i / w;
  dst[i] = src[r * s + c0 + (int)(i - r * w)];
}

void launch_gather_cols(int64_t n, int s, int c0, int w, const double* src, double* dst,
                        cudaStream_t st, pint_ctx ctx) {
  ProfScope ps(ctx, PF_VEC, 16.0 * n * w, 0.0, st);
  k_gather_cols<<<grid_for(n * w, 256), 256, 0, st>>>(n, s, c0, w, src, dst);
  check_launch("k_gather_cols");
  ctx->launches += 1;
}

// dst = src / colscale (per column); dst float64 or float32 (round to nearest)
template <typename OT>
__global__ void k_scale_cast(int64_t n, int s, const double* __restrict__ src, OT* __restrict__ dst,
                             const double* __restrict__ colnorm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * s) return;
  const int k = (int)(i % s);
  const double c = colnorm ? colnorm[k] : 1.0;
  const double v = c > 0.0 ? src[i] * (1.0 / c) : 0.0;
  if constexpr (std::is_same<OT, double>::value) dst[i] = v;
  else dst[i] = __double2float_rn(v);
}

void launch_scale_cast(int64_t n, int s, const double* src, float* dst, const double* colnorm,
                       cudaStream_t st, pint_ctx ctx) {
  ProfScope ps(ctx, PF_VEC, 12.0 * n * s, 1.0 * n * s, st);
  k_scale_cast<float><<<grid_for(n * s, 256), 256, 0, st>>>(n, s, src, dst, colnorm);
  check_launch("k_scale_cast");
  ctx->launches += 1;
}

void launch_scale_copy64(int64_t n, int s, const double* src, double* dst, const double* colnorm,
                         cudaStream_t st, pint_ctx ctx) {
  ProfScope ps(ctx, PF_VEC, 16.0 * n * s, 1.0 * n * s, st);
  k_scale_cast<double><<<grid_for(n * s, 256), 256, 0, st>>>(n, s, src, dst, colnorm);
  check_launch("k_scale_copy64");
  ctx->launches += 1;
}

void launch_copy_cast(int precision, int64_t n, int s, const double* src, void* dst,
                      cudaStream_t st, pint_ctx ctx) {
  if (precision == PINT_FP64)
    k_scale_cast<double><<<grid_for(n * s, 256), 256, 0, st>>>(n, s, src, (double*)dst, nullptr);
  else
    k_scale_cast<float><<<grid_for(n * s, 256), 256, 0, st>>>(n, s, src, (float*)dst, nullptr);
  check_launch("k_copy_cast");
  ctx->launches += 1;
}

// ---------------------------------------------------------------- shift
__global__ void k_shift(int64_t n, int s, double* __restrict__ Y) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double* y = Y + r * s;
  for (int k = 0; k + 1 < s; ++k) y[k] = y[k + 1];
}

void launch_shift(double* Y, int64_t n, int s, cudaStream_t st, pint_ctx ctx) {
  ProfScope ps(ctx, PF_VEC, 16.0 * n * s, 0.0, st);
  k_shift<<<grid_for(n, 256), 256, 0, st>>>(n, s, Y);
  check_launch("k_shift");
  if (ctx) ctx->launches += 1;
}

}  // namespace pint

namespace pint {
// ------------------------------------------------ Newton step bound
// out[k] = rnorm[k] * min(1, delta / max_r |rnorm[k] * rowscale[r] * X[r][k]|)
// The column maxima use atomicMax on the bit patterns of non-negative
// doubles (their integer order equals their numeric order): deterministic.
template <typename VT>
__global__ void k_colmax(int64_t n, int s, const VT* __restrict__ X,
                         const double* __restrict__ rowscale,
                         unsigned long long* __restrict__ bits) {
  double m[kMaxS];
  for (int k = 0; k < s; ++k) m[k] = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double rs = rowscale ? fabs(rowscale[r]) : 1.0;
    for (int k = 0; k < s; ++k) m[k] = fmax(m[k], rs * fabs((double)X[r * s + k]));
  }
  for (int k = 0; k < s; ++k) {
    double v = m[k];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(bits + k, (unsigned long long)__double_as_longlong(v));
  }
}

__global__ void k_step_scale(int s, const double* __restrict__ rnorm,
                             const unsigned long long* __restrict__ bits, double delta,
                             double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k >= s) return;
  const double step = rnorm[k] * __longlong_as_double((long long)bits[k]);
  out[k] = rnorm[k] * (step > delta ? delta / step : 1.0);
}

void launch_step_bound(int precision, int64_t n, int s, const void* X, const double* rowscale,
                       const double* rnorm, double delta, double* out, cudaStream_t st,
                       pint_ctx ctx) {
  unsigned long long* bits =
      reinterpret_cast<unsigned long long*>(ctx->d_small + kSmallScratch + 64);
  PINT_CUDA(cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * kMaxS, st));
  ProfScope ps(ctx, PF_VEC, (precision == PINT_FP64 ? 8.0 : 4.0) * n * s, 2.0 * n * s, st);
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ctx->num_sms * 4LL,
                                                                      (n + 255) / 256));
  if (precision == PINT_FP64)
    k_colmax<double><<<g, 256, 0, st>>>(n, s, (const double*)X, rowscale, bits);
  else
    k_colmax<float><<<g, 256, 0, st>>>(n, s, (const float*)X, rowscale, bits);
  k_step_scale<<<1, 32, 0, st>>>(s, rnorm, bits, delta, out);
  check_launch("k_colmax");
  ctx->launches += 2;
}
}  // namespace pint

namespace pint {
void bounds_take_spmm(unsigned long long* out) { pint_bounds_take(out); }
}  // namespace pint
