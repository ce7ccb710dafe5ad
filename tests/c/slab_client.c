/* A plain C client of libpint: one slab of s = 4 implicit-Euler steps of a
 * convection-diffusion operator on an 8 x 8 x 8 grid, through the C ABI
 * only (device buffers from the CUDA runtime, no Python). Prints the status,
 * the iteration counts and the largest column residual. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "pint.h"

int main(void) {
  enum { NX = 8, N = NX * NX * NX, S = 4 };
  const double tau = 1e-2;
  double* D = malloc(sizeof(double) * N);
  double* B = malloc(sizeof(double) * N * S);
  double A1[S * S] = {0}, A2[S * S] = {0};
  for (int i = 0; i < N; ++i) D[i] = 1.0 + 0.5 * sin(0.1 * i);
  for (int i = 0; i < N * S; ++i) B[i] = cos(0.37 * i);
  for (int k = 0; k < S; ++k) {              /* (I - L) / tau and I */
    A1[k * S + k] = 1.0 / tau;
    if (k > 0) A1[k * S + k - 1] = -1.0 / tau;
    A2[k * S + k] = 1.0;
  }
  pint_ctx ctx;
  pint_op op;
  if (pint_create(&ctx, 0, 0) != PINT_OK) {
    printf("create failed\n");
    return 1;
  }
  int rc = pint_fv_convdiff(ctx, &op, NX, NX, NX, D, 1.0, 0.5, 0.0, PINT_MEM_HOST, NULL);
  if (rc == PINT_OK) rc = pint_set_coupling(op, S, A1, A2);
  double *dB = NULL, *dY = NULL;
  if (rc == PINT_OK) {
    cudaMalloc((void**)&dB, sizeof(double) * N * S);
    cudaMalloc((void**)&dY, sizeof(double) * N * S);
    cudaMemcpy(dB, B, sizeof(double) * N * S, cudaMemcpyHostToDevice);
    cudaMemset(dY, 0, sizeof(double) * N * S);
    pint_opts o;
    pint_stats st;
    pint_opts_default(&o);
    o.tol = 1e-12;
    o.precond = PINT_PC_ILU0;
    rc = pint_solve_block(op, dB, NULL, dY, &o, &st, NULL);
    double worst = 0.0;
    for (int k = 0; k < S; ++k) worst = st.col_relres[k] > worst ? st.col_relres[k] : worst;
    printf("status %d outer %d inner %d max_relres %.3e\n", rc, st.outer_its, st.inner_its,
           worst);
    cudaFree(dB);
    cudaFree(dY);
    pint_operator_destroy(op);
  } else {
    printf("setup failed: %s\n", pint_last_error(ctx));
  }
  pint_destroy(ctx);
  free(D);
  free(B);
  return rc == PINT_OK ? 0 : 2;
}
