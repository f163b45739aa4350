/*
 * A C caller of the library's C ABI with no Python in the way: builds the
 * 16x16 lid-driven cavity hierarchy (3 levels) for the element given on the
 * command line (0 Q2-Q1, 1 stabilised Q1-Q1 with beta 0.02), sets up the
 * restricted additive Vanka smoother (Eq. 13; damping 0.5 on Q2-Q1, 0.66 on
 * Q1-Q1), solves to a 1e-8 residual reduction by stationary V(2,2) cycles and
 * by FGMRES, and prints "stationary <iterations> <ratio> fgmres <iterations>
 * <ratio>".  Device memory for x and b comes from the CUDA runtime; every
 * library call's status is checked.  Exit status 0 on success.
 */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "ravanka.h"

#define CHECK(call)                                                             \
  do {                                                                          \
    int rc_ = (call);                                                           \
    if (rc_ != RAV_OK) {                                                        \
      fprintf(stderr, "%s failed: %d (%s)\n", #call, rc_, rav_strerror(rc_));   \
      return 1;                                                                 \
    }                                                                           \
  } while (0)

int main(int argc, char** argv) {
  const int element = argc > 1 ? atoi(argv[1]) : RAV_ELEM_Q2Q1;
  rav_problem p = {0};
  p.dim = 2;
  p.N = 16;
  p.eta0 = 1.0;
  p.bc = RAV_BC_CAVITY;
  p.element = element;
  p.beta = 0.02;
  rav_mg* mg = NULL;
  rav_smoother* sm = NULL;
  CHECK(mg_setup(&p, 3, NULL, &mg));
  CHECK(vanka_setup(mg, RAV_RAV, RAV_F64, element == RAV_ELEM_Q1Q1 ? 0.66 : 0.5, NULL, &sm));
  int64_t counts[5];
  CHECK(rav_get_counts(mg, 2, counts));
  const size_t bytes = sizeof(double) * (size_t)counts[2];
  double *x = NULL, *b = NULL;
  if (cudaMalloc((void**)&x, bytes) != cudaSuccess || cudaMalloc((void**)&b, bytes) != cudaSuccess) {
    fprintf(stderr, "cudaMalloc failed\n");
    return 1;
  }
  CHECK(rav_assemble_rhs(mg, RAV_F_NONE, b, NULL));
  rav_solve_opts o = {1e-8, 100, 2, 2, 0, 30, 1e6, 0.0};
  rav_solve_info info[2];
  for (int outer = 0; outer < 2; ++outer) {
    CHECK(rav_initial_guess(mg, x, NULL));
    o.outer = outer;
    info[outer].history_host = NULL;
    CHECK(solve(mg, sm, x, b, &o, &info[outer], NULL));
  }
  printf("stationary %d %.3e fgmres %d %.3e\n", info[0].iterations, info[0].final_ratio, info[1].iterations,
         info[1].final_ratio);
  cudaFree(x);
  cudaFree(b);
  vanka_destroy(sm);
  mg_destroy(mg);
  return 0;
}
