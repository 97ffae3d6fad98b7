// Interface of the one-CTA FP64 Rayleigh-Ritz solver shared by the LOBPCG driver.
#pragma once
#include <cuda_runtime.h>

#define RR_MMAX 96
#define RR_KMAX 32

// G: [2][m][m] (G_A then G_B, row stride m).  Outputs: C [m][k] (coefficients of the k
// lowest Ritz vectors in the basis of G, rows past m_nop are 0 when P was dropped),
// theta [k] ascending, optional theta_hist [k] copy, optional Cp [m][k] (coefficients
// of the next P, B-orthogonal to the Ritz vectors).  *status must be 0 on entry
// (nonzero: the kernel does nothing); it becomes 2 for a dependent basis that dropping P
// does not cure and 3 for a non-finite Ritz value.  *restarts (optional) counts drops.
struct RRParams {
  const double* G;
  int m, k, m_nop;
  double* C;
  double* Cp;
  double* theta;
  double* theta_hist;
  int* status;
  int* restarts;
};

int bf_rr_launch(const RRParams& a, cudaStream_t s);
