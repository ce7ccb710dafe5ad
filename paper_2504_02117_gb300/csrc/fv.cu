// Cell-centred finite-volume workloads on [0,1]^d (h = 1/nx, x-fastest
// numbering), assembled and evaluated on the device, and the nonlinear
// drivers built on them: the simplified-Newton step and the pipelined window
// loop of Algorithm 1 (Sec. 2.2, Eq. matrix-equation-pipelining).
//
// Discretisation choices (the paper uses CCFV / Q1 FE and leaves these open):
// harmonic face means of the diffusion coefficient / K_S, homogeneous
// Dirichlet ghosts at h/2, first-order upwind convection with zero inflow;
// diffusion-reaction with the arithmetic face mean of (1+u^2) and zero-flux
// boundary; Richards with the upwind relative permeability by total head
// psi + z (tie: the lower cell index) and the van Genuchten-Mualem relations
// of Eq. RelationshipsThetaK read with theta/theta_S.
#include "internal.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

struct pint_problem_s {
  pint_ctx ctx = nullptr;
  int kind = 0;
  int nx = 1, ny = 1, nz = 1;
  int64_t n = 0;
  double vg_a = 1, vg_n = 2, vg_m = 0.5, th_r = 0.05, th_s = 0.4, dt_D = 1.0 / 16;
  double* Ks = nullptr;
  pint_op op = nullptr;
  double* scratch = nullptr;     // 2 n s doubles (theta, kr) for Richards
  size_t scratch_bytes = 0;
  double* vec = nullptr;         // n doubles
  double* B0 = nullptr;          // n * 16 window B0
  double* mstore = nullptr;      // converged stages: mass and f values
  double* fstore = nullptr;
  size_t store_cols = 0;
};

namespace pint {

void op_free_all(pint_op op);           // api.cu
void op_clear_inner_cache(pint_op op);  // api.cu

struct Grid {
  int nx, ny, nz;
  double h, ih2;
};

// ----------------------------------------------------------- stencil pattern
static void grid_pattern(int nx, int ny, int nz, std::vector<int>& rp, std::vector<int>& ci) {
  const int64_t n = (int64_t)nx * ny * nz;
  rp.assign(n + 1, 0);
  ci.clear();
  ci.reserve(n * 7);
  const int64_t sxy = (int64_t)nx * ny;
  for (int64_t r = 0; r < n; ++r) {
    const int i = (int)(r % nx), j = (int)((r / nx) % ny), k = (int)(r / sxy);
    if (k > 0) ci.push_back((int)(r - sxy));
    if (j > 0) ci.push_back((int)(r - nx));
    if (i > 0) ci.push_back((int)(r - 1));
    ci.push_back((int)r);
    if (i + 1 < nx) ci.push_back((int)(r + 1));
    if (j + 1 < ny) ci.push_back((int)(r + nx));
    if (k + 1 < nz) ci.push_back((int)(r + sxy));
    rp[r + 1] = (int)ci.size();
  }
}

// neighbour d in 0..5 = (-z, -y, -x, +x, +y, +z); returns -1 at the boundary
__device__ __forceinline__ int64_t nbr(const Grid& g, int64_t r, int i, int j, int k, int d) {
  const int64_t sxy = (int64_t)g.nx * g.ny;
  switch (d) {
    case 0: return g.nz > 1 && k > 0 ? r - sxy : -1;
    case 1: return g.ny > 1 && j > 0 ? r - g.nx : -1;
    case 2: return g.nx > 1 && i > 0 ? r - 1 : -1;
    case 3: return g.nx > 1 && i + 1 < g.nx ? r + 1 : -1;
    case 4: return g.ny > 1 && j + 1 < g.ny ? r + g.nx : -1;
    default: return g.nz > 1 && k + 1 < g.nz ? r + sxy : -1;
  }
}
// does direction d exist in this grid (for boundary faces)?
__device__ __forceinline__ bool has_dir(const Grid& g, int d) {
  return (d == 0 || d == 5) ? g.nz > 1 : (d == 1 || d == 4) ? g.ny > 1 : g.nx > 1;
}

// -------------------------------------------------- linear conv-diffusion
// Row r of K for -div(D grad u) + div(v u); CSR columns sorted (-z,-y,-x,P,+x,+y,+z).
__global__ void k_convdiff_values(Grid g, int64_t n, const double* __restrict__ D, double vx,
                                  double vy, double vz, const int* __restrict__ rowptr,
                                  double* __restrict__ K) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int i = (int)(r % g.nx), j = (int)((r / g.nx) % g.ny),
            k = (int)(r / ((int64_t)g.nx * g.ny));
  const double v[3] = {vx, vy, vz};
  const double DP = D[r];
  double diag = 0.0;
  double off[6] = {0, 0, 0, 0, 0, 0};
  for (int d = 0; d < 6; ++d) {
    if (!has_dir(g, d)) continue;
    const int ax = (d == 0 || d == 5) ? 2 : (d == 1 || d == 4) ? 1 : 0;
    const double sgn = d < 3 ? -1.0 : 1.0;
    const double vn = sgn * v[ax];           // outward normal velocity
    const int64_t q = nbr(g, r, i, j, k, d);
    if (q >= 0) {
      const double DQ = D[q];
      const double gf = (2.0 * DP * DQ / (DP + DQ)) * g.ih2;
      diag += gf;
      off[d] -= gf;
      if (vn > 0.0) diag += vn / g.h;
      else off[d] += vn / g.h;
    } else {
      diag += 2.0 * DP * g.ih2;
      if (vn > 0.0) diag += vn / g.h;
    }
  }
  int p = rowptr[r];
  for (int d = 0; d < 3; ++d)
    if (nbr(g, r, i, j, k, d) >= 0) K[p++] = off[d];
  K[p++] = diag;
  for (int d = 3; d < 6; ++d)
    if (nbr(g, r, i, j, k, d) >= 0) K[p++] = off[d];
}

// ---------------------------------------------------- van Genuchten-Mualem
struct Soil {
  double a, n, m, tr, ts;
};
__device__ __forceinline__ double vg_theta(const Soil& s, double psi) {
  if (psi > 0.0) return s.ts;
  const double u = pow(-s.a * psi, s.n);
  return s.tr + (s.ts - s.tr) * pow(1.0 + u, -s.m);
}
__device__ __forceinline__ double vg_dtheta(const Soil& s, double psi) {
  if (psi >= 0.0) return 0.0;
  const double x = -s.a * psi;
  return (s.ts - s.tr) * s.m * s.n * s.a * pow(x, s.n - 1.0) * pow(1.0 + pow(x, s.n), -s.m - 1.0);
}
__device__ __forceinline__ double vg_kr(const Soil& s, double psi) {
  const double x = vg_theta(s, psi) / s.ts;
  const double w = fmax(1.0 - pow(x, 1.0 / s.m), 0.0);
  const double b = 1.0 - pow(w, s.m);
  return sqrt(x) * b * b;
}
__device__ __forceinline__ double vg_dkr(const Soil& s, double psi) {
  const double x = vg_theta(s, psi) / s.ts;
  const double w = 1.0 - pow(x, 1.0 / s.m);
  if (!(psi < 0.0) || !(w > 1e-12)) return 0.0;
  const double b = 1.0 - pow(w, s.m);
  const double dkdx = 0.5 / sqrt(x) * b * b + sqrt(x) * 2.0 * b * pow(w, s.m - 1.0) *
                                                   pow(x, 1.0 / s.m - 1.0);
  return dkdx / s.ts * vg_dtheta(s, psi);
}

struct NlParams {
  int kind;
  Soil soil;
  const double* Ks;
  double cx[kMaxS];      // diffreact: circle centre x per column
  double psiD[kMaxS];    // richards: Dirichlet head per column
};

__device__ __forceinline__ bool top_patch(const Grid& g, int i, int j, int k) {
  return k == g.nz - 1 && (i + 0.5) * g.h < 0.5 && (j + 0.5) * g.h < 0.5;
}

// Richards pointwise pass: theta and kr per cell and column.
template <int S, bool EXACT>
__global__ void k_rich_point(int64_t n, int s, Soil soil, const double* __restrict__ Y,
                             double* __restrict__ TH, double* __restrict__ KR) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double y[S], th[S], kr[S];
  load_row<S, EXACT>(Y + r * s, s, y);
#pragma unroll
  for (int c = 0; c < S; ++c) {
    th[c] = vg_theta(soil, y[c]);
    kr[c] = vg_kr(soil, y[c]);
  }
  store_row<S, EXACT>(TH + r * s, s, th);
  store_row<S, EXACT>(KR + r * s, s, kr);
}

// R_r = M(Y)_r A1^T + F(T,Y)_r A2^T - B0_r (Eq. matrix-equation-pipelining
// residual) with the column-wise nonlinear f evaluated from the stencil.
template <int S, bool EXACT, int LO>
__global__ void __launch_bounds__(128)
k_nl_residual(Grid g, int64_t n, int s, const __grid_constant__ NlParams P,
              const double* __restrict__ Y, const double* __restrict__ TH,
              const double* __restrict__ KR, const double* __restrict__ B0,
              double* __restrict__ R, const __grid_constant__ Coupling cp) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int i = (int)(r % g.nx), j = (int)((r / g.nx) % g.ny),
            k = (int)(r / ((int64_t)g.nx * g.ny));
  double y[S], f[S], mass[S];
  load_row<S, EXACT>(Y + r * s, s, y);
  if (P.kind == PINT_PROBLEM_DIFFREACT) {
    const double x = (i + 0.5) * g.h, yy = (j + 0.5) * g.h;
#pragma unroll
    for (int c = 0; c < S; ++c) {
      const double dx = x - P.cx[c], dy = yy - 0.5;
      const double src = (dx * dx + dy * dy <= 0.01) ? -0.1 : 0.0;
      f[c] = -y[c] * (1.0 - y[c]) - src;
      mass[c] = y[c];
    }
    for (int d = 0; d < 6; ++d) {
      const int64_t q = nbr(g, r, i, j, k, d);
      if (q < 0) continue;
      double yq[S];
      load_row<S, EXACT>(Y + q * s, s, yq);
#pragma unroll
      for (int c = 0; c < S; ++c) {
        const double a = 1.0 + 0.5 * (y[c] * y[c] + yq[c] * yq[c]);
        f[c] -= a * (yq[c] - y[c]) * g.ih2;
      }
    }
  } else {
    const double zP = (k + 0.5) * g.h;
    const double KsP = P.Ks[r];
    double krP[S];
    load_row<S, EXACT>(TH + r * s, s, mass);
    load_row<S, EXACT>(KR + r * s, s, krP);
#pragma unroll
    for (int c = 0; c < S; ++c) f[c] = 0.0;
    for (int d = 0; d < 6; ++d) {
      const int64_t q = nbr(g, r, i, j, k, d);
      if (q < 0) continue;
      const double KsQ = P.Ks[q];
      const double kf = 2.0 * KsP * KsQ / (KsP + KsQ);
      const double zQ = (d == 0) ? zP - g.h : (d == 5) ? zP + g.h : zP;
      double yq[S], krQ[S];
      load_row<S, EXACT>(Y + q * s, s, yq);
      load_row<S, EXACT>(KR + q * s, s, krQ);
#pragma unroll
      for (int c = 0; c < S; ++c) {
        const double HP = y[c] + zP, HQ = yq[c] + zQ;
        const bool upQ = (HQ > HP) || (HQ == HP && q < r);
        const double K = kf * (upQ ? krQ[c] : krP[c]);
        f[c] -= K * (HQ - HP) * g.ih2;
      }
    }
    if (top_patch(g, i, j, k)) {
#pragma unroll
      for (int c = 0; c < S; ++c) {
        const double HP = y[c] + zP, HD = P.psiD[c] + 1.0;
        const double K = KsP * (HD > HP ? vg_kr(P.soil, P.psiD[c]) : krP[c]);
        f[c] -= 2.0 * K * (HD - HP) * g.ih2;
      }
    }
  }
  double out[S];
  if (B0) {
    load_row<S, EXACT>(B0 + r * s, s, out);
#pragma unroll
    for (int c = 0; c < S; ++c) out[c] = -out[c];
  } else {
#pragma unroll
    for (int c = 0; c < S; ++c) out[c] = 0.0;
  }
#pragma unroll
  for (int a = 0; a < S; ++a) {
    if (!EXACT && a >= s) break;
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < S; ++c) {
      if (!EXACT && c >= s) break;
      if (LO > 0 && (c > a || a - c > LO)) continue;
      const double a1 = cp.A1[a * kMaxS + c];
      const double a2 = cp.A2[a * kMaxS + c];
      if (LO > 0) {
        acc = fma(a1, mass[c], acc);
        acc = fma(a2, f[c], acc);
      } else {
        if (a1 != 0.0) acc = fma(a1, mass[c], acc);
        if (a2 != 0.0) acc = fma(a2, f[c], acc);
      }
    }
    out[a] += acc;
  }
  store_row<S, EXACT>(R + r * s, s, out);
}

// One column: mass and f (used for B0 terms of converged stages).
__global__ void k_nl_eval(Grid g, int64_t n, const __grid_constant__ NlParams P,
                          const double* __restrict__ y, double* __restrict__ mout,
                          double* __restrict__ fout) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int i = (int)(r % g.nx), j = (int)((r / g.nx) % g.ny),
            k = (int)(r / ((int64_t)g.nx * g.ny));
  const double yp = y[r];
  double f = 0.0, m = yp;
  if (P.kind == PINT_PROBLEM_DIFFREACT) {
    const double dx = (i + 0.5) * g.h - P.cx[0], dy = (j + 0.5) * g.h - 0.5;
    f = -yp * (1.0 - yp) - ((dx * dx + dy * dy <= 0.01) ? -0.1 : 0.0);
    for (int d = 0; d < 6; ++d) {
      const int64_t q = nbr(g, r, i, j, k, d);
      if (q < 0) continue;
      const double a = 1.0 + 0.5 * (yp * yp + y[q] * y[q]);
      f -= a * (y[q] - yp) * g.ih2;
    }
  } else {
    const double zP = (k + 0.5) * g.h, KsP = P.Ks[r];
    const double krP = vg_kr(P.soil, yp);
    m = vg_theta(P.soil, yp);
    for (int d = 0; d < 6; ++d) {
      const int64_t q = nbr(g, r, i, j, k, d);
      if (q < 0) continue;
      const double kf = 2.0 * KsP * P.Ks[q] / (KsP + P.Ks[q]);
      const double zQ = (d == 0) ? zP - g.h : (d == 5) ? zP + g.h : zP;
      const double HP = yp + zP, HQ = y[q] + zQ;
      const bool upQ = (HQ > HP) || (HQ == HP && q < r);
      f -= kf * (upQ ? vg_kr(P.soil, y[q]) : krP) * (HQ - HP) * g.ih2;
    }
    if (top_patch(g, i, j, k)) {
      const double HP = yp + zP, HD = P.psiD[0] + 1.0;
      f -= 2.0 * KsP * (HD > HP ? vg_kr(P.soil, P.psiD[0]) : krP) * (HD - HP) * g.ih2;
    }
  }
  if (mout) mout[r] = m;
  if (fout) fout[r] = f;
}

// Row r of J = alpha M'(y) + beta Df(t, y) in the stencil CSR order; y is
// column 0 of a row-major N x ys block. Also writes diag(J) and its inverse.
//
// Richards with lsL > 0: the L-scheme matrix alpha lsL I + beta A(y), A the
// flux operator with the conductivities frozen at y (kr not differentiated).
__global__ void k_nl_jacobian(Grid g, int64_t n, const __grid_constant__ NlParams P,
                              const double* __restrict__ Y, int ys, double alpha, double beta,
                              double lsL,
                              const int* __restrict__ rowptr, double* __restrict__ J,
                              double* __restrict__ Jd, double* __restrict__ Jinv) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int i = (int)(r % g.nx), j = (int)((r / g.nx) % g.ny),
            k = (int)(r / ((int64_t)g.nx * g.ny));
  const double yp = Y[r * ys];
  double diag, off[6] = {0, 0, 0, 0, 0, 0};
  if (P.kind == PINT_PROBLEM_DIFFREACT) {
    diag = alpha - beta * (1.0 - 2.0 * yp);
    for (int d = 0; d < 6; ++d) {
      const int64_t q = nbr(g, r, i, j, k, d);
      if (q < 0) continue;
      const double yq = Y[q * ys];
      const double a = 1.0 + 0.5 * (yp * yp + yq * yq);
      const double du = yq - yp;
      diag += beta * (a - yp * du) * g.ih2;
      off[d] = -beta * (a + yq * du) * g.ih2;
    }
  } else {
    const Soil& so = P.soil;
    const double zP = (k + 0.5) * g.h, KsP = P.Ks[r];
    const bool frozen = lsL > 0.0;
    const double krP = vg_kr(so, yp), dkrP = frozen ? 0.0 : vg_dkr(so, yp);
    diag = frozen ? alpha * lsL : alpha * vg_dtheta(so, yp);
    for (int d = 0; d < 6; ++d) {
      const int64_t q = nbr(g, r, i, j, k, d);
      if (q < 0) continue;
      const double yq = Y[q * ys];
      const double kf = 2.0 * KsP * P.Ks[q] / (KsP + P.Ks[q]);
      const double zQ = (d == 0) ? zP - g.h : (d == 5) ? zP + g.h : zP;
      const double HP = yp + zP, HQ = yq + zQ;
      const bool upQ = (HQ > HP) || (HQ == HP && q < r);
      const double K = kf * (upQ ? vg_kr(so, yq) : krP);
      const double dKQ = (upQ && !frozen) ? kf * vg_dkr(so, yq) : 0.0;
      const double dKP = upQ ? 0.0 : kf * dkrP;
      const double dH = HQ - HP;
      diag += beta * (K - dKP * dH) * g.ih2;
      off[d] = -beta * (K + dKQ * dH) * g.ih2;
    }
    if (top_patch(g, i, j, k)) {
      const double HP = yp + zP, HD = P.psiD[0] + 1.0;
      const bool up = HD > HP;
      const double K = KsP * (up ? vg_kr(so, P.psiD[0]) : krP);
      const double dK = up ? 0.0 : KsP * dkrP;
      diag += beta * 2.0 * (K - dK * (HD - HP)) * g.ih2;
    }
  }
  int p = rowptr[r];
  for (int d = 0; d < 3; ++d)
    if (nbr(g, r, i, j, k, d) >= 0) J[p++] = off[d];
  J[p++] = diag;
  for (int d = 3; d < 6; ++d)
    if (nbr(g, r, i, j, k, d) >= 0) J[p++] = off[d];
  Jd[r] = diag;
  Jinv[r] = 1.0 / diag;
}

// B0[:, col] += coef * v
__global__ void k_b0_axpy(int64_t n, int s, int col, double coef, const double* __restrict__ v,
                          double* __restrict__ B0) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) B0[r * s + col] += coef * v[r];
}

// dst[r*ds + dc] = src[r*ss + sc]
__global__ void k_copy_col(int64_t n, const double* __restrict__ src, int ss, int sc,
                           double* __restrict__ dst, int ds, int dc) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) dst[r * ds + dc] = src[r * ss + sc];
}

static Grid grid_of(const pint_problem p) {
  return Grid{p->nx, p->ny, p->nz, 1.0 / p->nx, (double)p->nx * p->nx};
}

static NlParams params_of(const pint_problem p, const double* times, int s) {
  NlParams P;
  std::memset(&P, 0, sizeof(P));
  P.kind = p->kind;
  P.soil = Soil{p->vg_a, p->vg_n, p->vg_m, p->th_r, p->th_s};
  P.Ks = p->Ks;
  for (int c = 0; c < s; ++c) {
    const double t = times[c];
    P.cx[c] = 0.5 + 0.25 * std::cos(6.0 * t);
    P.psiD[c] = t <= p->dt_D ? -2.0 + 2.2 * t / p->dt_D : 0.2;
  }
  return P;
}

static void nl_residual(pint_problem p, const double* times, const double* Y, const double* B0,
                        double* R, cudaStream_t st) {
  pint_op op = p->op;
  const int s = op->s;
  const int64_t n = p->n;
  NlParams P = params_of(p, times, s);
  Grid g = grid_of(p);
  Coupling cp;
  std::copy(op->A1, op->A1 + kMaxS * kMaxS, cp.A1);
  std::copy(op->A2, op->A2 + kMaxS * kMaxS, cp.A2);
  double* TH = nullptr;
  double* KR = nullptr;
  if (p->kind == PINT_PROBLEM_RICHARDS) {
    const size_t need = 2 * sizeof(double) * n * s;
    if (p->scratch_bytes < need) {
      dfree(p->ctx, p->scratch, p->scratch_bytes);
      p->scratch = (double*)dalloc(p->ctx, need);
      p->scratch_bytes = need;
    }
    TH = p->scratch;
    KR = p->scratch + n * s;
  }
  ProfScope ps(p->ctx, PF_COUPLED,
               8.0 * n * s * (2 + (B0 ? 1 : 0) + (p->kind == PINT_PROBLEM_RICHARDS ? 4 : 0)),
               30.0 * n * s, st);
  with_s(s, [&](auto S_, auto E_) {
    constexpr int S = decltype(S_)::value;
    constexpr bool E = decltype(E_)::value;
    if (p->kind == PINT_PROBLEM_RICHARDS) {
      k_rich_point<S, E><<<grid_for(n, 128), 128, 0, st>>>(n, s, P.soil, Y, TH, KR);
      p->ctx->launches += 1;
    }
    const int lo = coupling_band(op->A1, op->A2, s);
    auto launch = [&](auto kern) {
      kern<<<grid_for(n, 128), 128, 0, st>>>(g, n, s, P, Y, TH, KR, B0, R, cp);
    };
    if (lo == 1) launch(k_nl_residual<S, E, 1>);
    else if (lo == 2) launch(k_nl_residual<S, E, 2>);
    else launch(k_nl_residual<S, E, 0>);
  });
  check_launch("k_nl_residual");
  p->ctx->launches += 1;
}

static void nl_eval(pint_problem p, double t, const double* y, double* m, double* f,
                    cudaStream_t st) {
  NlParams P = params_of(p, &t, 1);
  ProfScope ps(p->ctx, PF_NL, 24.0 * p->n, 30.0 * p->n, st);
  k_nl_eval<<<grid_for(p->n, 128), 128, 0, st>>>(grid_of(p), p->n, P, y, m, f);
  check_launch("k_nl_eval");
  p->ctx->launches += 1;
}

// sup over psi of theta'(psi) for van Genuchten: with x = alpha |psi|,
// theta' = (ts - tr) m n alpha x^(n-1) (1 + x^n)^(-m-1), stationary where
// (n-1)(1 + x^n) = (m+1) n x^n, i.e. x^n = (n-1)/(mn+1) = m for m = 1 - 1/n.
static double vg_lipschitz(double a, double n, double tr, double ts) {
  const double m = 1.0 - 1.0 / n;
  const double x = std::pow(m, 1.0 / n);
  return (ts - tr) * m * n * a * std::pow(x, n - 1.0) * std::pow(1.0 + m, -m - 1.0);
}

static void nl_jacobian(pint_problem p, double t, const double* Y, int ys, double lsL,
                        cudaStream_t st) {
  pint_op op = p->op;
  op_clear_inner_cache(op);
  if (!op->Jval) {
    op->Jval = dalloc_n<double>(op->ctx, op->nnz);
    op->Jdiag = dalloc_n<double>(op->ctx, op->n);
    op->Jinvdiag = dalloc_n<double>(op->ctx, op->n);
  }
  NlParams P = params_of(p, &t, 1);
  ProfScope ps(p->ctx, PF_NL, 8.0 * op->nnz + 24.0 * p->n, 60.0 * p->n, st);
  k_nl_jacobian<<<grid_for(p->n, 128), 128, 0, st>>>(grid_of(p), p->n, P, Y, ys, op->alpha,
                                                     op->beta, lsL, op->rowptr, op->Jval,
                                                     op->Jdiag, op->Jinvdiag);
  check_launch("k_nl_jacobian");
  p->ctx->launches += 1;
  op->j_valid = true;
}

static double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// One simplified-Newton iteration (body of the inner loop of Algorithm 1):
// R = R(Y); stop if ||R_0|| <= tol ||B0_0||; J = alpha M'(Y_0) + beta Df(t_0, Y_0);
// solve J V = R for all s columns; Y <- Y - V.
static void newton_step(pint_problem p, const double* times, double* Y, const double* B0,
                        const pint_opts* o, int* converged, pint_stats* stats, cudaStream_t st) {
  PINT_REQUIRE(std::isfinite(o->lscheme_L) &&
                   (o->lscheme_L == 0.0 || p->kind == PINT_PROBLEM_RICHARDS),
               PINT_ERR_INVALID, "the L-scheme (lscheme_L != 0) applies to Richards problems");
  PINT_REQUIRE(o->solver >= PINT_SOLVER_GMRES && o->solver <= PINT_SOLVER_BICGSTAB,
               PINT_ERR_INVALID, "solver");
  pint_op op = p->op;
  pint_ctx ctx = p->ctx;
  const int s = op->s;
  const int64_t n = p->n;
  double* R = nullptr;
  double* rnorm = nullptr;
  void* Xk = nullptr;
  int wprec = 0;
  work_views(op, o->precision == PINT_FP64 ? PINT_FP64 : PINT_FP32, o->restart, &R, &rnorm, &Xk,
             &wprec);
  nl_residual(p, times, Y, B0, R, st);
  launch_colnorm(ctx, PINT_FP64, n, s, R, rnorm, st);
  double* b0n = ctx->d_small + kSmallScratch;
  if (B0) {
    launch_colnorm(ctx, PINT_FP64, n, s, B0, b0n, st);
    PINT_CUDA(cudaMemcpyAsync(ctx->h_small + 64, b0n, 8 * s, cudaMemcpyDeviceToHost, st));
  }
  PINT_CUDA(cudaMemcpyAsync(ctx->h_small, rnorm, 8 * s, cudaMemcpyDeviceToHost, st));
  PINT_CUDA(cudaStreamSynchronize(st));
  const double f0 = B0 ? ctx->h_small[64] : 0.0;
  const double r0 = ctx->h_small[0];
  const double scale = f0 > 0.0 ? f0 : 1.0;
  {
    double rel[kMaxS];
    for (int k = 0; k < s; ++k) rel[k] = ctx->h_small[k] / scale;
    hist_push(ctx, rel, s);
    if (stats)
      for (int k = 0; k < s; ++k) stats->col_relres[k] = rel[k];
  }
  for (int k = 0; k < s; ++k)
    PINT_REQUIRE(std::isfinite(ctx->h_small[k]), PINT_ERR_BREAKDOWN, "non-finite Newton residual");
  if (r0 <= o->tol * scale) {
    *converged = 1;
    return;
  }
  *converged = 0;
  double lsL = o->lscheme_L;
  if (lsL < 0.0) lsL = vg_lipschitz(p->vg_a, p->vg_n, p->th_r, p->th_s);
  nl_jacobian(p, times[0], Y, s, lsL, st);
  const double ts = now_ms();
  if (o->precond == PINT_PC_ILU0) ilu_setup(op, st);
  if (stats) stats->setup_ms += now_ms() - ts;
  InnerResult ir = inner_solve(op, o, R, rnorm, nullptr, st);
  if (stats) {
    stats->inner_its += ir.its;
    stats->restarts += ir.cycles;
    stats->deflations += ir.deflations;
  }
  // block GMRES with Jacobi solves for D V (see solve_block_impl); CG for V
  const double* rs =
      o->precond == PINT_PC_JACOBI && o->solver != PINT_SOLVER_CG ? op->Jinvdiag : nullptr;
  const double* cs = rnorm;
  if (o->max_step > 0.0) {
    double* bounded = ctx->d_small + kSmallScratch + 128;
    launch_step_bound(wprec, n, s, Xk, rs, rnorm, o->max_step, bounded, st, ctx);
    cs = bounded;
  }
  launch_outer_update(wprec, n, s, Y, Xk, cs, rs, st, ctx);
}

// Window of s consecutive stages starting at global stage g0 (0-based) of the
// stiffly accurate DIRK (A, c): A1, A2 and the B0 recipe (Eq. matrix-equation-
// pipelining with the known stages moved to B0). Stage (n, k) reads
// (1/tau)(M(y^{(n,k)}) - M(y^n)) + sum_{j<=k} a_kj f_j = 0, y^n = y^{(n-1,m)}.
struct Term {
  int col;
  int kind;   // 0: mass of stage g, 1: f of stage g
  int g;      // global stage (-1: the initial value)
  double coef;
};

static void window(const double* A, const double* c, int m, double tau, int g0, int s,
                   double* A1, double* A2, std::vector<Term>& terms, double* times) {
  std::fill(A1, A1 + s * s, 0.0);
  std::fill(A2, A2 + s * s, 0.0);
  terms.clear();
  for (int i = 0; i < s; ++i) {
    const int g = g0 + i;
    const int nstep = g / m, k = g % m + 1;
    times[i] = (nstep + c[k - 1]) * tau;
    A1[i * s + i] += 1.0 / tau;
    const int gprev = nstep * m - 1;
    if (gprev >= g0) A1[i * s + (gprev - g0)] += -1.0 / tau;
    else terms.push_back({i, 0, gprev, 1.0 / tau});
    for (int jj = 1; jj <= k; ++jj) {
      const int gj = nstep * m + jj - 1;
      const double a = A[(k - 1) * m + (jj - 1)];
      if (gj >= g0) A2[i * s + (gj - g0)] += a;
      else if (a != 0.0) terms.push_back({i, 1, gj, -a});
    }
  }
}

static void set_window_coupling(pint_op op, int s, const double* A1, const double* A2) {
  const int rc = pint_set_coupling(op, s, A1, A2);
  if (rc != PINT_OK) throw Error{rc, op->ctx->err};
}

static void ensure_store(pint_problem p, int cols) {
  if ((int)p->store_cols >= cols) return;
  const size_t old = p->store_cols;
  dfree(p->ctx, p->mstore, sizeof(double) * p->n * old);
  dfree(p->ctx, p->fstore, sizeof(double) * p->n * old);
  p->mstore = dalloc_n<double>(p->ctx, p->n * cols);
  p->fstore = dalloc_n<double>(p->ctx, p->n * cols);
  p->store_cols = cols;
}

}  // namespace pint

using namespace pint;

namespace {
template <typename Fn>
int guard_p(pint_ctx ctx, Fn&& fn) {
  try {
    if (ctx) PINT_CUDA(cudaSetDevice(ctx->device));
    return fn();
  } catch (const Error& e) {
    if (ctx) ctx->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->err = "host allocation failed";
    return PINT_ERR_NOMEM;
  }
}
}  // namespace

extern "C" {

int pint_fv_convdiff(pint_ctx ctx, pint_op* out, int nx, int ny, int nz, const double* D,
                     double vx, double vy, double vz, int mem_space, void* stream) {
  if (!ctx || !out) return PINT_ERR_INVALID;
  *out = nullptr;
  return guard_p(ctx, [&] {
    PINT_REQUIRE(nx >= 1 && ny >= 1 && nz >= 1 && D, PINT_ERR_INVALID, "grid");
    PINT_REQUIRE(mem_space == PINT_MEM_HOST || mem_space == PINT_MEM_DEVICE, PINT_ERR_INVALID,
                 "mem_space");
    const int64_t n = (int64_t)nx * ny * nz;
    PINT_REQUIRE(n < (int64_t)1 << 30, PINT_ERR_INVALID, "grid too large");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<int> rp, ci;
    grid_pattern(nx, ny, nz, rp, ci);
    pint_op op = op_create(ctx, n, rp.data(), ci.data(), st);
    op->grid_nx = nx;
    op->grid_ny = ny;
    op->grid_nz = nz;
    try {
      const double* dD = D;
      double* tmp = nullptr;
      if (mem_space == PINT_MEM_HOST) {
        tmp = dalloc_n<double>(ctx, n);
        PINT_CUDA(cudaMemcpyAsync(tmp, D, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        dD = tmp;
      }
      Grid g{nx, ny, nz, 1.0 / nx, (double)nx * nx};
      k_convdiff_values<<<grid_for(n, 256), 256, 0, st>>>(g, n, dD, vx, vy, vz, op->rowptr,
                                                          op->Kval);
      check_launch("k_convdiff_values");
      ctx->launches += 1;
      sell_scatter(op, op->Kval, op->sellK, st);
      PINT_CUDA(cudaStreamSynchronize(st));
      if (tmp) dfree(ctx, tmp, sizeof(double) * n);
    } catch (...) {
      op_free_all(op);
      delete op;
      throw;
    }
    *out = op;
    return PINT_OK;
  });
}

int pint_problem_create(pint_ctx ctx, pint_problem* out, int kind, int nx, int ny, int nz,
                        const double* params, const double* field, void* stream) {
  if (!ctx || !out) return PINT_ERR_INVALID;
  *out = nullptr;
  return guard_p(ctx, [&] {
    PINT_REQUIRE(kind == PINT_PROBLEM_DIFFREACT || kind == PINT_PROBLEM_RICHARDS,
                 PINT_ERR_INVALID, "problem kind");
    PINT_REQUIRE(nx >= 1 && ny >= 1 && nz >= 1, PINT_ERR_INVALID, "grid");
    const int64_t n = (int64_t)nx * ny * nz;
    PINT_REQUIRE(n < (int64_t)1 << 30, PINT_ERR_INVALID, "grid too large");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    pint_problem p = new pint_problem_s();
    p->ctx = ctx;
    p->kind = kind;
    p->nx = nx;
    p->ny = ny;
    p->nz = nz;
    p->n = n;
    try {
      if (kind == PINT_PROBLEM_RICHARDS) {
        PINT_REQUIRE(params && field, PINT_ERR_INVALID, "Richards needs params and K_S");
        p->vg_a = params[0];
        p->vg_n = params[1];
        p->th_r = params[2];
        p->th_s = params[3];
        p->dt_D = params[4];
        PINT_REQUIRE(p->vg_n > 1.0 && p->vg_a > 0.0 && p->th_s > p->th_r && p->dt_D > 0.0,
                     PINT_ERR_INVALID, "van Genuchten parameters");
        p->vg_m = (p->vg_n - 1.0) / p->vg_n;
        p->Ks = dalloc_n<double>(ctx, n);
        PINT_CUDA(cudaMemcpyAsync(p->Ks, field, sizeof(double) * n, cudaMemcpyDefault, st));
      }
      std::vector<int> rp, ci;
      grid_pattern(nx, ny, nz, rp, ci);
      p->op = op_create(ctx, n, rp.data(), ci.data(), st);
      p->op->grid_nx = nx;
      p->op->grid_ny = ny;
      p->op->grid_nz = nz;
      p->op->owner = p;
      p->vec = dalloc_n<double>(ctx, n);
      p->B0 = dalloc_n<double>(ctx, n * kMaxS);
      PINT_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
      pint_problem_destroy(p);
      throw;
    }
    *out = p;
    return PINT_OK;
  });
}

int pint_vg_lipschitz(const double* params, double* L) {
  if (!params || !L) return PINT_ERR_INVALID;
  const double a = params[0], n = params[1], tr = params[2], ts = params[3];
  if (!(n > 1.0) || !(a > 0.0) || !(ts > tr)) return PINT_ERR_INVALID;
  *L = vg_lipschitz(a, n, tr, ts);
  return PINT_OK;
}

int pint_problem_destroy(pint_problem p) {
  if (!p) return PINT_ERR_INVALID;
  pint_ctx c = p->ctx;
  cudaSetDevice(c->device);
  if (p->op) {
    op_free_all(p->op);
    delete p->op;
  }
  dfree(c, p->Ks, sizeof(double) * p->n);
  dfree(c, p->scratch, p->scratch_bytes);
  dfree(c, p->vec, sizeof(double) * p->n);
  dfree(c, p->B0, sizeof(double) * p->n * kMaxS);
  dfree(c, p->mstore, sizeof(double) * p->n * p->store_cols);
  dfree(c, p->fstore, sizeof(double) * p->n * p->store_cols);
  delete p;
  return PINT_OK;
}

pint_op pint_problem_operator(pint_problem p) { return p ? p->op : nullptr; }

int pint_problem_eval(pint_problem p, double t, const double* y, double* mass_out,
                      double* f_out, void* stream) {
  if (!p) return PINT_ERR_INVALID;
  return guard_p(p->ctx, [&] {
    PINT_REQUIRE(y, PINT_ERR_INVALID, "NULL y");
    nl_eval(p, t, y, mass_out, f_out, static_cast<cudaStream_t>(stream));
    return PINT_OK;
  });
}

int pint_problem_residual(pint_problem p, const double* times, const double* Y,
                          const double* B0, double* R, void* stream) {
  if (!p) return PINT_ERR_INVALID;
  return guard_p(p->ctx, [&] {
    PINT_REQUIRE(p->op->s >= 1, PINT_ERR_INVALID, "coupling not set");
    PINT_REQUIRE(times && Y && R, PINT_ERR_INVALID, "NULL argument");
    PINT_REQUIRE(reinterpret_cast<uintptr_t>(Y) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(R) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(B0) % 16 == 0,
                 PINT_ERR_INVALID, "block vectors must be 16-byte aligned");
    nl_residual(p, times, Y, B0, R, static_cast<cudaStream_t>(stream));
    return PINT_OK;
  });
}

int pint_newton_step(pint_problem p, const double* times, double* Y, const double* B0,
                     const pint_opts* opts, int* converged, pint_stats* stats, void* stream) {
  if (!p) return PINT_ERR_INVALID;
  pint_opts o;
  if (opts) o = *opts; else pint_opts_default(&o);
  if (stats) std::memset(stats, 0, sizeof(*stats));
  const long l0 = p->ctx->launches;
  const double t0 = now_ms();
  int rc = guard_p(p->ctx, [&] {
    PINT_REQUIRE(p->op->s >= 1, PINT_ERR_INVALID, "coupling not set");
    PINT_REQUIRE(times && Y && converged, PINT_ERR_INVALID, "NULL argument");
    PINT_REQUIRE(reinterpret_cast<uintptr_t>(Y) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(B0) % 16 == 0,
                 PINT_ERR_INVALID, "block vectors must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    newton_step(p, times, Y, B0, &o, converged, stats, st);
    PINT_CUDA(cudaStreamSynchronize(st));
    return PINT_OK;
  });
  if (stats) {
    stats->status = rc;
    stats->outer_its = 1;
    stats->solve_ms = now_ms() - t0;
    stats->kernel_launches = (int)(p->ctx->launches - l0);
  }
  return rc;
}

int pint_pipeline_run(pint_problem p, const double* A, const double* c, int m, double tau, int s,
                      const double* y0, int nstages, double* stages_out, const pint_opts* opts,
                      pint_stats* stats, void* stream) {
  if (!p) return PINT_ERR_INVALID;
  pint_opts o;
  if (opts) o = *opts; else pint_opts_default(&o);
  if (stats) std::memset(stats, 0, sizeof(*stats));
  const long l0 = p->ctx->launches;
  const double t0 = now_ms();
  int newton_total = 0;
  int rc = guard_p(p->ctx, [&] {
    hist_reset(p->ctx, s);
    PINT_REQUIRE(A && c && y0 && stages_out && m >= 1 && s >= 1 && s <= PINT_MAX_S &&
                     nstages >= 1 && tau > 0.0,
                 PINT_ERR_INVALID, "bad arguments");
    for (int k = 0; k < m; ++k)
      PINT_REQUIRE(A[k * m + k] != 0.0, PINT_ERR_INVALID,
                   "every stage must be implicit (a_kk != 0)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = p->n;
    pint_op op = p->op;
    ensure_store(p, nstages + 1);      // column 0: the initial value
    // window state Y and its B0 (N x s each)
    double* Ybuf = dalloc_n<double>(p->ctx, n * s);
    double* Bbuf = dalloc_n<double>(p->ctx, n * s);
    try {
      for (int k = 0; k < s; ++k)
        k_copy_col<<<grid_for(n, 256), 256, 0, st>>>(n, y0, 1, 0, Ybuf, s, k);
      check_launch("k_copy_col");
      // stored mass of y0 in column 0 of mstore (f unused for the initial value)
      nl_eval(p, 0.0, y0, p->mstore, nullptr, st);
      double A1[kMaxS * kMaxS], A2[kMaxS * kMaxS], times[kMaxS];
      std::vector<Term> terms;
      for (int g0 = 0; g0 < nstages; ++g0) {
        window(A, c, m, tau, g0, s, A1, A2, terms, times);
        set_window_coupling(op, s, A1, A2);
        PINT_CUDA(cudaMemsetAsync(Bbuf, 0, sizeof(double) * n * s, st));
        for (const Term& t : terms) {
          const double* v = t.kind == 0 ? p->mstore + (size_t)(t.g + 1) * n
                                        : p->fstore + (size_t)(t.g + 1) * n;
          k_b0_axpy<<<grid_for(n, 256), 256, 0, st>>>(n, s, t.col, t.coef, v, Bbuf);
        }
        check_launch("k_b0_axpy");
        p->ctx->launches += (long)terms.size();
        int conv = 0, it = 0;
        for (it = 0; it <= o.max_outer; ++it) {
          newton_step(p, times, Ybuf, Bbuf, &o, &conv, stats, st);
          if (conv) break;
        }
        PINT_REQUIRE(conv, PINT_ERR_NOT_CONVERGED,
                     "Newton did not converge in window " + std::to_string(g0));
        newton_total += it;
        k_copy_col<<<grid_for(n, 256), 256, 0, st>>>(n, Ybuf, s, 0, stages_out, nstages, g0);
        k_copy_col<<<grid_for(n, 256), 256, 0, st>>>(n, Ybuf, s, 0, p->vec, 1, 0);
        check_launch("k_copy_col");
        p->ctx->launches += 2;
        nl_eval(p, times[0], p->vec, p->mstore + (size_t)(g0 + 1) * n,
                p->fstore + (size_t)(g0 + 1) * n, st);
        if (s > 1) launch_shift(Ybuf, n, s, st, p->ctx);
      }
      PINT_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
      dfree(p->ctx, Ybuf, sizeof(double) * n * s);
      dfree(p->ctx, Bbuf, sizeof(double) * n * s);
      throw;
    }
    dfree(p->ctx, Ybuf, sizeof(double) * n * s);
    dfree(p->ctx, Bbuf, sizeof(double) * n * s);
    return PINT_OK;
  });
  if (stats) {
    stats->status = rc;
    stats->outer_its = newton_total;
    stats->solve_ms = now_ms() - t0;
    stats->kernel_launches = (int)(p->ctx->launches - l0);
  }
  return rc;
}

}  // extern "C"
